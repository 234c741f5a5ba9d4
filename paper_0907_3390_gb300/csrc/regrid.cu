// regrid.cu -- the rebuild of the refinement map on the device (Sec. 2.1
// step 4): the flag step over one level and the data of a rebuilt level.
// Compiled with -fmad=false: the criteria are evaluated in FP64 in the
// order of their plain definition, so that flags never depend on the
// precision of the handle or on contraction.
#include "common.cuh"
#include "internal.h"

namespace gh {

// Quantity of the criterion at one cell (density, or the pressure of Eqs.
// ThermalEnergy, EOS with v = m / rho), in FP64.
template <typename T>
__device__ __forceinline__ double crit_q(const T* __restrict__ u, size_t vs, size_t off, int criterion,
                                         double gamma) {
    const double rho = (double)u[off];
    if (criterion != 1) return rho;
    const double vx = (double)u[vs + off] / rho;
    const double vy = (double)u[2 * vs + off] / rho;
    const double vz = (double)u[3 * vs + off] / rho;
    const double eps = (double)u[4 * vs + off] - 0.5 * rho * (vx * vx + vy * vy + vz * vz);
    return (gamma - 1.0) * eps;
}

constexpr int NT_FLAG = 512;

// One block per patch group.  A cell is flagged by criterion 0 / 1 when
// the largest relative change of density / pressure across one cell width,
// |q(+1) - q(-1)| / (2 |q|) over the three axes, reaches the threshold
// (Eqs. ShockTube_RefineCriterion, BlastWave_RefineCriterion; a neighbour
// that only exists on the coarser level counts as the cell itself), and by
// criterion 2 when rho exceeds the threshold.  Its flag buffer, the cube of
// 1 + 2 n_buffer cells around it, sets in its patch's mask the bit of every
// patch offset (dx,dy,dz) it reaches: (dz+1)*9 + (dy+1)*3 + (dx+1).
template <typename T>
__global__ void __launch_bounds__(NT_FLAG) k_flag(const FlagArgs<T> a) {
    __shared__ int s_src[27], s_mask[27];
    __shared__ unsigned s_m[8];
    const int g = blockIdx.x, t = threadIdx.x;
    if (t < 27) region_entry(a.nbr, g, t, s_src, s_mask);
    if (t < 8) s_m[t] = 0u;
    __syncthreads();
    const size_t vs = (size_t)a.n_groups * 8 * 512;
    for (int i = t; i < CELLS_PG; i += NT_FLAG) {
        const int x = i % GS, y = (i / GS) % GS, z = i / (GS * GS);
        const double q0 = crit_q(a.u, vs, cell_offset(g, x, y, z), a.criterion == 2 ? 0 : a.criterion, a.gamma);
        bool hit;
        if (a.criterion == 2) {
            hit = q0 > a.threshold;
        } else {
            double rmax = 0.0;
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                double q[2];
#pragma unroll
                for (int sd = 0; sd < 2; ++sd) {
                    int c[3] = {x, y, z};
                    c[ax] += sd == 0 ? -1 : 1;
                    const int src = resolve(s_src, s_mask, c[0], c[1], c[2]);
                    q[sd] = src < 0 ? q0 : crit_q(a.u, vs, cell_offset(src, c[0], c[1], c[2]), a.criterion, a.gamma);
                }
                const double r = fabs(q[1] - q[0]) / (2.0 * fabs(q0));
                if (r > rmax) rmax = r;
            }
            hit = rmax >= a.threshold;
        }
        if (!hit) continue;
        const int pc[3] = {x % PS, y % PS, z % PS};
        int lo[3], hi[3];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            lo[ax] = pc[ax] - a.n_buffer < 0 ? -1 : 0;
            hi[ax] = pc[ax] + a.n_buffer > PS - 1 ? 1 : 0;
        }
        unsigned m = 0u;
        for (int dz = lo[2]; dz <= hi[2]; ++dz)
            for (int dy = lo[1]; dy <= hi[1]; ++dy)
                for (int dx = lo[0]; dx <= hi[0]; ++dx) m |= 1u << ((dz + 1) * 9 + (dy + 1) * 3 + (dx + 1));
        atomicOr(&s_m[((z / PS) * 2 + (y / PS)) * 2 + (x / PS)], m);
    }
    __syncthreads();
    if (t < 8) a.masks[8 * g + t] = s_m[t];
}

template <typename T>
cudaError_t launch_flag(const FlagArgs<T>& a, cudaStream_t st) {
    if (a.n_groups <= 0) return cudaSuccess;
    k_flag<T><<<a.n_groups, NT_FLAG, 0, st>>>(a);
    return cudaGetLastError();
}
template cudaError_t launch_flag<float>(const FlagArgs<float>&, cudaStream_t);
template cudaError_t launch_flag<double>(const FlagArgs<double>&, cudaStream_t);

constexpr int NT_REF = 256;

// One block per group of the rebuilt level: a copy of the old group it
// inherits, or every cell by Min-Mod interpolation from its parent patch
// on the level below (the refinement step of Sec. 2.1).
template <typename T>
__global__ void __launch_bounds__(NT_REF) k_refine(const RefineArgs<T> a) {
    __shared__ int s_csrc[27], s_cmask[27];
    const int g = blockIdx.x, t = threadIdx.x;
    const size_t vs = (size_t)a.n_new * 8 * 512;
    const int src = a.inherit[g];
    if (src >= 0) {
        const size_t vso = (size_t)a.n_old * 8 * 512;
        for (int v = 0; v < NV; ++v) {
            const float4* in = reinterpret_cast<const float4*>(a.u_old + v * vso + (size_t)src * CELLS_PG);
            float4* out = reinterpret_cast<float4*>(a.u_new + v * vs + (size_t)g * CELLS_PG);
            constexpr int N4 = CELLS_PG * (int)sizeof(T) / 16;
            for (int i = t; i < N4; i += NT_REF) out[i] = in[i];
        }
        return;
    }
    const int P = a.parent_new[g];
    if (t < 27) region_entry(a.nbrc, P >> 3, t, s_csrc, s_cmask);
    __syncthreads();
    const size_t vsc = (size_t)a.n_c * 8 * 512;
    for (int i = t; i < CELLS_PG; i += NT_REF) {
        const int x = i % GS, y = (i / GS) % GS, z = i / (GS * GS);
        T val[NV];
        prolong<T>(a.uc, nullptr, T(0), vsc, s_csrc, s_cmask, P & 1, (P >> 1) & 1, (P >> 2) & 1, x, y, z, val);
        const size_t off = cell_offset(g, x, y, z);
#pragma unroll
        for (int v = 0; v < NV; ++v) a.u_new[v * vs + off] = val[v];
    }
}

template <typename T>
cudaError_t launch_refine(const RefineArgs<T>& a, cudaStream_t st) {
    if (a.n_new <= 0) return cudaSuccess;
    k_refine<T><<<a.n_new, NT_REF, 0, st>>>(a);
    return cudaGetLastError();
}
template cudaError_t launch_refine<float>(const RefineArgs<float>&, cudaStream_t);
template cudaError_t launch_refine<double>(const RefineArgs<double>&, cudaStream_t);

}  // namespace gh
