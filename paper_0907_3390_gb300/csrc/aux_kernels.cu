// aux_kernels.cu -- coarse-fine fix-up and diagnostics (CFL maxima,
// conservation sums, positivity count), for both element types.
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace gh {

// ------------------------------------------------------------ fix-up

// One thread block of 512 threads per listed coarse patch P (one thread per
// cell of the 8^3 patch).  A refined patch (child >= 0) gets the mean of
// its 8 children per cell (restriction, Sec. 2.1 step 3); a leaf patch gets
// the coarse-fine flux correction on every face whose same-level neighbour
// patch is refined: the coarse flux is replaced by the mean of the 4 fine
// fluxes of that face (Berger-Colella), faces in the order x-, x+, y-, y+,
// z-, z+.
template <typename T>
__global__ void __launch_bounds__(512) k_fixup(const FixArgs<T> a) {
    using V2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
    __shared__ double s_lam;
    if (threadIdx.x == 0) s_lam = (*a.dt * a.dts) / a.dh;   // coarse lambda = dt / dh
    __syncthreads();
    const T lam = (T)s_lam;
    const int P = a.list[blockIdx.x];
    const int g = P >> 3, lp = P & 7;
    const int pc[3] = {lp & 1, (lp >> 1) & 1, (lp >> 2) & 1};
    const int t = threadIdx.x;
    const int ci[3] = {t & 7, (t >> 3) & 7, t >> 6};
    const size_t vsc = (size_t)a.n_c * 8 * 512, vsf = (size_t)a.n_f * 8 * 512;
    const int X = PS * pc[0] + ci[0], Y = PS * pc[1] + ci[1], Z = PS * pc[2] + ci[2];
    const size_t co = cell_offset(g, X, Y, Z);
    const int gf = a.child[P];
    if (gf >= 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const T* f = a.uf + v * vsf;
            T s = T(0);
#pragma unroll
            for (int dz = 0; dz < 2; ++dz)
#pragma unroll
                for (int dy = 0; dy < 2; ++dy) {
                    // the two x-children in one aligned load, added in order
                    const V2 c = *reinterpret_cast<const V2*>(f + cell_offset(gf, 2 * ci[0], 2 * ci[1] + dy,
                                                                               2 * ci[2] + dz));
                    s = s + c.x;
                    s = s + c.y;
                }
            a.uc[v * vsc + co] = T(0.125) * s;
        }
        return;
    }
    T val[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) val[v] = a.uc[v * vsc + co];
    bool touched = false;
    for (int ax = 0; ax < 3; ++ax) {
        const int t1 = ax == 0 ? 1 : 0, t2 = ax == 2 ? 1 : 2;
        for (int s = -1; s <= 1; s += 2) {
            if (ci[ax] != (s > 0 ? PS - 1 : 0)) continue;
            int q[3] = {pc[0], pc[1], pc[2]};
            q[ax] += s;
            int gq = g;
            if (q[ax] < 0 || q[ax] > 1) {
                int e[3] = {0, 0, 0};
                e[ax] = s;
                gq = a.nbr[(size_t)g * 26 + dir_index(e[0], e[1], e[2])];
                q[ax] = q[ax] < 0 ? 1 : 0;
            }
            if (gq < 0) continue;
            const int gfq = a.child[8 * gq + (q[2] * 2 + q[1]) * 2 + q[0]];
            if (gfq < 0) continue;
            const int plane_c = s > 0 ? pc[ax] + 1 : pc[ax];
            const int plane_f = s > 0 ? 0 : 2;
            const int b1 = ci[t1], b2 = ci[t2];
            const int T1 = PS * pc[t1] + b1, T2 = PS * pc[t2] + b2;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const T Gc = a.flux_c[((((size_t)g * 3 + ax) * 3 + plane_c) * NV + v) * 256 + T2 * GS + T1];
                const size_t fo = ((((size_t)gfq * 3 + ax) * 3 + plane_f) * NV + v) * 256;
                const size_t k00 = fo + (2 * b2) * GS + 2 * b1, k01 = k00 + 1, k10 = k00 + GS, k11 = k10 + 1;
                T f00 = a.flux_f[k00], f01 = a.flux_f[k01], f10 = a.flux_f[k10], f11 = a.flux_f[k11];
                if (a.flux_f2 != nullptr) {
                    // individual time steps: mean over the finer level's two steps
                    f00 = T(0.5) * (f00 + a.flux_f2[k00]);
                    f01 = T(0.5) * (f01 + a.flux_f2[k01]);
                    f10 = T(0.5) * (f10 + a.flux_f2[k10]);
                    f11 = T(0.5) * (f11 + a.flux_f2[k11]);
                }
                const T Gf = T(0.25) * (((f00 + f01) + f10) + f11);
                if (s > 0) val[v] = val[v] + lam * (Gc - Gf);
                else val[v] = val[v] - lam * (Gc - Gf);
            }
            touched = true;
        }
    }
    if (touched) {
#pragma unroll
        for (int v = 0; v < NV; ++v) a.uc[v * vsc + co] = val[v];
    }
}

template <typename T>
cudaError_t launch_fixup(const FixArgs<T>& a, int n_list, cudaStream_t st) {
    if (n_list <= 0) return cudaSuccess;
    k_fixup<T><<<n_list, 512, 0, st>>>(a);
    return cudaGetLastError();
}
template cudaError_t launch_fixup<float>(const FixArgs<float>&, int, cudaStream_t);
template cudaError_t launch_fixup<double>(const FixArgs<double>&, int, cudaStream_t);

// ------------------------------------------------------------ diagnostics

// Signal speed c_s + max(|vx|,|vy|,|vz|) of one cell (denominator of Eq.
// CFL) and its pressure.  FP64: the plain order of operations; FP32: the
// fast single-precision forms of the FP32 path.
__device__ __forceinline__ void speed_pressure(const double u[NV], double g, double gm1, double& s,
                                               double& P) {
    const double rho = u[0];
    const double vx = u[1] / rho, vy = u[2] / rho, vz = u[3] / rho;
    const double eps = u[4] - (0.5 * rho) * ((vx * vx + vy * vy) + vz * vz);
    P = gm1 * eps;
    const double cs = sqrt((g * fmax(P, 0.0)) / rho);
    s = cs + fmax(fmax(fabs(vx), fabs(vy)), fabs(vz));
}
__device__ __forceinline__ void speed_pressure(const float u[NV], float g, float gm1, float& s,
                                               float& P) {
    speed_pressure_f32(u, g, gm1, s, P);
}

// Error-free accumulation for the FP32 path: a double-float (hi, lo) pair
// per thread (Knuth's two-sum), converted to FP64 before any cross-thread
// combination.  The FP64 path accumulates in FP64 directly.
struct Acc32 {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float s = hi + x;
        const float bb = s - hi;
        const float err = (hi - (s - bb)) + (x - bb);
        hi = s;
        lo += err;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};
struct Acc64 {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double value() const { return s; }
};
template <typename T> struct AccOf;
template <> struct AccOf<float> { using type = Acc32; };
template <> struct AccOf<double> { using type = Acc64; };

constexpr int NT_DIAG = 256;

// One block per patch group (of any level): exact per-group maximum of the
// signal speed over all cells, leaf-cell sums of the 5 conserved variables
// (fixed assignment of cells to threads, fixed tree) and the count of leaf
// cells with rho <= 0, P <= 0 or a non-finite variable.
template <typename T>
__global__ void __launch_bounds__(NT_DIAG) k_diag(const DiagArgs<T> a) {
    using Acc = typename AccOf<T>::type;
    const int item = blockIdx.x;
    int l = 0;
    while (l + 1 < a.n_levels && item >= a.lv[l + 1].item0) ++l;
    const DiagLevel<T>& L = a.lv[l];
    const int g = item - L.item0;
    const size_t vstride = (size_t)L.n_groups * 8 * 512;
    const T* base = L.u + ((size_t)g << 12);
    // the speed maximum as the bit pattern of a non-negative T (a NaN wins),
    // widened to double once per thread
    using Bits = typename std::conditional<sizeof(T) == 4, unsigned, unsigned long long>::type;
    Bits smax_t = 0;
    Acc acc[NV];
    int bad = 0;
    // one cell of the group (fixed assignment of cells to threads)
    auto cell = [&](const T u[NV], bool leaf) {
        bool finite = true;
#pragma unroll
        for (int v = 0; v < NV; ++v) finite = finite && isfinite(u[v]);
        T s, P;
        speed_pressure(u, a.gamma, a.gm1, s, P);
        Bits sb;
        memcpy(&sb, &s, sizeof(T));
        smax_t = sb > smax_t ? sb : smax_t;
        if (leaf) {
#pragma unroll
            for (int v = 0; v < NV; ++v) acc[v].add(u[v]);
            if (!finite || !(u[0] > T(0)) || !(P > T(0))) ++bad;
        }
    };
    if constexpr (sizeof(T) == 4) {
        // FP32: thread t takes the aligned quads t, t + 256, ... (all 20 of
        // its 16-byte loads in flight before the first cell is formed)
        constexpr int NQ = CELLS_PG / 4 / NT_DIAG;
        float4 w[NQ][NV];
#pragma unroll
        for (int k = 0; k < NQ; ++k)
#pragma unroll
            for (int v = 0; v < NV; ++v)
                w[k][v] = __ldg(reinterpret_cast<const float4*>(base + v * vstride) + threadIdx.x + k * NT_DIAG);
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
            const int patch = (threadIdx.x + k * NT_DIAG) >> 7;      // 128 quads per patch
            const bool leaf = L.child == nullptr || L.child[8 * g + patch] < 0;
            T u[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) u[v] = w[k][v].x;
            cell(u, leaf);
#pragma unroll
            for (int v = 0; v < NV; ++v) u[v] = w[k][v].y;
            cell(u, leaf);
#pragma unroll
            for (int v = 0; v < NV; ++v) u[v] = w[k][v].z;
            cell(u, leaf);
#pragma unroll
            for (int v = 0; v < NV; ++v) u[v] = w[k][v].w;
            cell(u, leaf);
        }
    } else {
#pragma unroll 4
        for (int i = threadIdx.x; i < CELLS_PG; i += NT_DIAG) {
            const int patch = i >> 9;
            const bool leaf = L.child == nullptr || L.child[8 * g + patch] < 0;
            T u[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) u[v] = base[v * vstride + i];
            cell(u, leaf);
        }
    }
    T smax_v;
    memcpy(&smax_v, &smax_t, sizeof(T));
    const unsigned long long smax = (unsigned long long)__double_as_longlong((double)smax_v);
    __shared__ double s_sum[NV][NT_DIAG];
    __shared__ unsigned long long s_max[NT_DIAG];
    __shared__ int s_bad[NT_DIAG];
#pragma unroll
    for (int v = 0; v < NV; ++v) s_sum[v][threadIdx.x] = acc[v].value();
    s_max[threadIdx.x] = smax;
    s_bad[threadIdx.x] = bad;
    __syncthreads();
    for (int w = NT_DIAG / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
#pragma unroll
            for (int v = 0; v < NV; ++v) s_sum[v][threadIdx.x] += s_sum[v][threadIdx.x + w];
            s_max[threadIdx.x] = max(s_max[threadIdx.x], s_max[threadIdx.x + w]);
            s_bad[threadIdx.x] += s_bad[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.pg_max[item] = s_max[0];
#pragma unroll
        for (int v = 0; v < NV; ++v) a.pg_sum[(size_t)item * NV + v] = s_sum[v][0];
        a.pg_bad[item] = s_bad[0];
    }
}

// One block per level: combine the per-group results of the level in a
// fixed order (strided partials, then a fixed tree).
template <typename T>
__global__ void __launch_bounds__(NT_FIN) k_diag_final(const DiagArgs<T> a) {
    const int l = blockIdx.x;
    const int i0 = a.lv[l].item0, n = a.lv[l].n_groups;
    double sum[NV] = {0, 0, 0, 0, 0};
    unsigned long long m = 0ull;
    long long bad = 0;
    for (int i = threadIdx.x; i < n; i += NT_FIN) {
#pragma unroll
        for (int v = 0; v < NV; ++v) sum[v] += a.pg_sum[(size_t)(i0 + i) * NV + v];
        m = max(m, a.pg_max[i0 + i]);
        bad += a.pg_bad[i0 + i];
    }
    __shared__ double s_sum[NV][NT_FIN];
    __shared__ unsigned long long s_max[NT_FIN];
    __shared__ long long s_bad[NT_FIN];
#pragma unroll
    for (int v = 0; v < NV; ++v) s_sum[v][threadIdx.x] = sum[v];
    s_max[threadIdx.x] = m;
    s_bad[threadIdx.x] = bad;
    __syncthreads();
    for (int w = NT_FIN / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
#pragma unroll
            for (int v = 0; v < NV; ++v) s_sum[v][threadIdx.x] += s_sum[v][threadIdx.x + w];
            s_max[threadIdx.x] = max(s_max[threadIdx.x], s_max[threadIdx.x + w]);
            s_bad[threadIdx.x] += s_bad[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        DiagOut* o = a.out + l;
        o->smax_bits = s_max[0];
#pragma unroll
        for (int v = 0; v < NV; ++v) o->sum[v] = s_sum[v][0];
        o->n_bad = s_bad[0];
    }
}

template <typename T>
cudaError_t launch_diag(const DiagArgs<T>& a, int total, cudaStream_t st) {
    if (total > 0) {
        k_diag<T><<<total, NT_DIAG, 0, st>>>(a);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_diag_final<T><<<a.n_levels, NT_FIN, 0, st>>>(a);
    return cudaGetLastError();
}
template cudaError_t launch_diag<float>(const DiagArgs<float>&, int, cudaStream_t);
template cudaError_t launch_diag<double>(const DiagArgs<double>&, int, cudaStream_t);

template <typename T>
cudaError_t launch_diag_groups(const DiagArgs<T>& a, int total, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    k_diag<T><<<total, NT_DIAG, 0, st>>>(a);
    return cudaGetLastError();
}
template cudaError_t launch_diag_groups<float>(const DiagArgs<float>&, int, cudaStream_t);
template cudaError_t launch_diag_groups<double>(const DiagArgs<double>&, int, cudaStream_t);

// ------------------------------------------------------------ whole step

__global__ void k_set_dt(double* slot, double dt) { *slot = dt; }

cudaError_t launch_set_dt(double* slot, double dt, cudaStream_t st) {
    k_set_dt<<<1, 1, 0, st>>>(slot, dt);
    return cudaGetLastError();
}

// One block: the end-of-step reduction (step_reduce.cuh) as its own launch,
// for multi-level and FP64 steps.
__global__ void __launch_bounds__(NT_FIN) k_step_final(const LevelMeta m, const unsigned long long* pg_max,
                                                      const double* pg_sum, const int* pg_bad, double cfl,
                                                      double* dt, int update_dt, StepOut* out,
                                                      StepOut* out_host) {
    __shared__ double s_sum[NV * NT_FIN];
    __shared__ unsigned long long s_max[NT_FIN];
    __shared__ long long s_bad[NT_FIN];
    step_reduce(m, pg_max, pg_sum, pg_bad, cfl, dt, update_dt, out, out_host, nullptr, s_sum, s_max, s_bad);
}

cudaError_t launch_step_final(const DiagArgs<float>& a32, const DiagArgs<double>& a64, bool fp64,
                              const double* dh, const double* dscale, double cfl, double* dt, int update_dt,
                              StepOut* out, StepOut* out_host, cudaStream_t st) {
    LevelMeta m;
    m.n_levels = fp64 ? a64.n_levels : a32.n_levels;
    for (int l = 0; l < m.n_levels; ++l) {
        m.item0[l] = fp64 ? a64.lv[l].item0 : a32.lv[l].item0;
        m.n[l] = fp64 ? a64.lv[l].n_groups : a32.lv[l].n_groups;
        m.dh[l] = dh[l];
        m.dscale[l] = dscale ? dscale[l] : 1.0;
    }
    const unsigned long long* pm = fp64 ? a64.pg_max : a32.pg_max;
    const double* ps = fp64 ? a64.pg_sum : a32.pg_sum;
    const int* pb = fp64 ? a64.pg_bad : a32.pg_bad;
    k_step_final<<<1, NT_FIN, 0, st>>>(m, pm, ps, pb, cfl, dt, update_dt, out, out_host);
    return cudaGetLastError();
}

}  // namespace gh
