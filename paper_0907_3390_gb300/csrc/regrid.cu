// regrid.cu -- the rebuild of the refinement map on the device (Sec. 2.1
// step 4): the flag step over one level and the data of a rebuilt level.
// Compiled with -fmad=false: the criteria are evaluated in the order of
// their plain definition, in the handle's precision, so that flags never
// depend on contraction.
#include "common.cuh"
#include "internal.h"

namespace gh {

// Quantity of the criterion at one cell (density, or the pressure of Eqs.
// ThermalEnergy, EOS with v = m / rho), in the precision T of the state:
// single precision is the paper's GPU precision, and the flags of a
// single-precision run are decided in it.
template <typename T>
__device__ __forceinline__ T crit_q(const T* __restrict__ u, size_t vs, size_t off, int criterion, T gm1) {
    const T rho = u[off];
    if (criterion != 1) return rho;
    const T vx = u[vs + off] / rho;
    const T vy = u[2 * vs + off] / rho;
    const T vz = u[3 * vs + off] / rho;
    const T eps = u[4 * vs + off] - T(0.5) * rho * (vx * vx + vy * vy + vz * vz);
    return gm1 * eps;
}

constexpr int NT_FLAG = 512;
constexpr int HP = GS + 2;    // the group with one halo cell per side

// One block per patch group.  The criterion's quantity of the group and of
// its one-cell halo is evaluated once per cell into shared memory.  A cell
// is flagged by criterion 0 / 1 when the largest relative change of
// density / pressure across one cell width, |q(+1) - q(-1)| / (2 |q|) over
// the three axes, reaches the threshold (Eqs. ShockTube_RefineCriterion,
// BlastWave_RefineCriterion; a neighbour that only exists on the coarser
// level counts as the cell itself), and by criterion 2 when rho exceeds the
// threshold.  Its flag buffer, the cube of 1 + 2 n_buffer cells around it,
// sets in its patch's mask the bit of every patch offset (dx,dy,dz) it
// reaches: (dz+1)*9 + (dy+1)*3 + (dx+1).
template <typename T>
__global__ void __launch_bounds__(NT_FLAG) k_flag(const FlagArgs<T> a) {
    __shared__ T s_q[HP * HP * HP];
    __shared__ int s_src[27], s_mask[27];
    __shared__ unsigned s_m[8];
    const int g = blockIdx.x, t = threadIdx.x;
    if (t < 27) region_entry(a.nbr, g, t, s_src, s_mask);
    if (t < 8) s_m[t] = 0u;
    __syncthreads();
    const size_t vs = (size_t)a.n_groups * 8 * 512;
    const T gm1 = T(a.gamma - 1.0);
    const int crit = a.criterion == 2 ? 0 : a.criterion;
    // the group's own cells, in memory order (coalesced): local index j =
    // ((patch * 8 + z) * 8 + y) * 8 + x with patch = (pz * 2 + py) * 2 + px
    const size_t base = (size_t)g * CELLS_PG;
    for (int j = t; j < CELLS_PG; j += NT_FLAG) {
        const int p = j >> 9, x = ((p & 1) << 3) | (j & 7), y = (((p >> 1) & 1) << 3) | ((j >> 3) & 7),
                  z = ((p >> 2) << 3) | ((j >> 6) & 7);
        s_q[((z + 1) * HP + (y + 1)) * HP + (x + 1)] = crit_q<T>(a.u, vs, base + j, crit, gm1);
    }
    // the one-cell halo through the region table (the gradient criteria only)
    constexpr int NH = HP * HP * HP - CELLS_PG;
    for (int k = t; k < (a.criterion == 2 ? 0 : NH); k += NT_FLAG) {
        // k-th halo position: z = -1 and z = 16 planes, then per interior z
        // the y = -1 and y = 16 rows, then per interior (y, z) the two x ends
        int x, y, z;
        if (k < 2 * HP * HP) {
            z = k < HP * HP ? -1 : GS;
            const int r = k % (HP * HP);
            x = r % HP - 1;
            y = r / HP - 1;
        } else if (k < 2 * HP * HP + 2 * GS * HP) {
            const int r = k - 2 * HP * HP;
            z = r / (2 * HP);
            y = (r % (2 * HP)) < HP ? -1 : GS;
            x = r % HP - 1;
        } else {
            const int r = k - 2 * HP * HP - 2 * GS * HP;
            z = r / (2 * GS);
            y = (r % (2 * GS)) >> 1;
            x = (r & 1) ? GS : -1;
        }
        const int idx = ((z + 1) * HP + (y + 1)) * HP + (x + 1);
        const int src = resolve(s_src, s_mask, x, y, z);
        s_q[idx] = src < 0 ? T(0) : crit_q<T>(a.u, vs, cell_offset(src, x, y, z), crit, gm1);
    }
    __syncthreads();
    // cells in memory order: pass k covers patch k, so the masks of a pass
    // combine by warp reductions before one shared atomic per warp
#pragma unroll 1
    for (int k = 0; k < CELLS_PG / NT_FLAG; ++k) {
        const int j = k * NT_FLAG + t;
        const int p = j >> 9, x = ((p & 1) << 3) | (j & 7), y = (((p >> 1) & 1) << 3) | ((j >> 3) & 7),
                  z = ((p >> 2) << 3) | ((j >> 6) & 7);
        const int c0 = ((z + 1) * HP + (y + 1)) * HP + (x + 1);
        const T q0 = s_q[c0];
        bool hit;
        if (a.criterion == 2) {
            hit = (double)q0 > a.threshold;
        } else {
            T rmax = T(0);
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                const int st = ax == 0 ? 1 : ax == 1 ? HP : HP * HP;
                T q[2];
#pragma unroll
                for (int sd = 0; sd < 2; ++sd) {
                    int c[3] = {x, y, z};
                    c[ax] += sd == 0 ? -1 : 1;
                    const int r = (region_of(c[2]) + 1) * 9 + (region_of(c[1]) + 1) * 3 + (region_of(c[0]) + 1);
                    q[sd] = s_src[r] < 0 ? q0 : s_q[c0 + (sd == 0 ? -st : st)];
                }
                const T r = fabs(q[1] - q[0]) / (T(2) * fabs(q0));
                if (r > rmax) rmax = r;
            }
            hit = (double)rmax >= a.threshold;
        }
        unsigned m = 0u;
        if (hit) {
            // patch offsets the buffer reaches along each axis, as 3-bit sets
            // (bit d+1 for offset d), spread into the 27-bit mask
            const int pc[3] = {x & 7, y & 7, z & 7};
            unsigned sa[3];
#pragma unroll
            for (int ax = 0; ax < 3; ++ax)
                sa[ax] = 2u | (pc[ax] - a.n_buffer < 0 ? 1u : 0u) | (pc[ax] + a.n_buffer > PS - 1 ? 4u : 0u);
            const unsigned row = sa[0];
            const unsigned plane = ((sa[1] & 1u) ? row : 0u) | ((sa[1] & 2u) ? row << 3 : 0u) |
                                   ((sa[1] & 4u) ? row << 6 : 0u);
            m = ((sa[2] & 1u) ? plane : 0u) | ((sa[2] & 2u) ? plane << 9 : 0u) | ((sa[2] & 4u) ? plane << 18 : 0u);
        }
        m = __reduce_or_sync(0xffffffffu, m);
        if ((t & 31) == 0 && m != 0u) atomicOr(&s_m[p], m);
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
