// regrid.cu -- the rebuild of the refinement map on the device (Sec. 2.1
// step 4): the flag step over one level and the data of a rebuilt level.
// Compiled with -fmad=false: the criteria are evaluated in the order of
// their plain definition, in the handle's precision, so that flags never
// depend on contraction.
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace gh {

// Quantity of the criterion at one cell (density, or the pressure of Eqs.
// ThermalEnergy, EOS with v = m / rho), in the precision T of the state:
// single precision is the paper's GPU precision, and the flags of a
// single-precision run are decided in it.  Raw<T, QC> holds the values the
// quantity needs (QC = 1: pressure, all five variables; else density), so
// that their loads can be issued well before the quantity is formed.
template <typename T, int QC>
struct Raw {
    T r[QC == 1 ? NV : 1];
};

template <typename T, int QC>
__device__ __forceinline__ Raw<T, QC> load_raw(const T* __restrict__ u, size_t vs, size_t off) {
    Raw<T, QC> w;
#pragma unroll
    for (int v = 0; v < (QC == 1 ? NV : 1); ++v) w.r[v] = u[v * vs + off];
    return w;
}

template <typename T, int QC>
__device__ __forceinline__ T quantity(const Raw<T, QC>& w, T gm1) {
    const T rho = w.r[0];
    if (QC != 1) return rho;
    const T vx = w.r[QC == 1 ? 1 : 0] / rho;
    const T vy = w.r[QC == 1 ? 2 : 0] / rho;
    const T vz = w.r[QC == 1 ? 3 : 0] / rho;
    const T eps = w.r[QC == 1 ? 4 : 0] - T(0.5) * rho * (vx * vx + vy * vy + vz * vz);
    return gm1 * eps;
}

template <typename T>
__device__ __forceinline__ T crit_q(const T* __restrict__ u, size_t vs, size_t off, int criterion, T gm1) {
    return criterion == 1 ? quantity<T, 1>(load_raw<T, 1>(u, vs, off), gm1)
                          : quantity<T, 0>(load_raw<T, 0>(u, vs, off), gm1);
}

constexpr int NT_FLAG = 512;
// resident blocks per SM: as many as the registers of the prefetched next
// group allow (8 values per thread, 40 for the pressure)
template <typename T, int CRIT>
constexpr int flag_blocks_per_sm() {
    return sizeof(T) == 4 ? (CRIT == 1 ? 2 : CRIT == 0 ? 3 : 4) : (CRIT == 1 ? 1 : 2);
}
constexpr int HP = GS + 2;    // the group with one halo cell per side
// shared-memory pitches of the staged quantity: a warp tests 4 rows of 8
// cells of one plane; in single precision a row pitch of 24 words puts the
// 4 rows on disjoint banks (with 18 they overlap); double precision keeps
// 18, which holds the block within the 48 KB of static shared memory
template <typename T>
struct SqPitch {
    static constexpr int RW = sizeof(T) == 4 ? 24 : HP;
    static constexpr int PLN = HP * RW;
    static __device__ __forceinline__ int index(int x, int y, int z) {
        return (z + 1) * PLN + (y + 1) * RW + (x + 1);
    }
};
constexpr int PER_FLAG = CELLS_PG / NT_FLAG;   // interior cells per thread

// The flag step.  A cell is flagged by criterion 0 / 1 when the largest
// relative change of density / pressure across one cell width,
// |q(+1) - q(-1)| / (2 |q|) over the three axes, reaches the threshold
// (Eqs. ShockTube_RefineCriterion, BlastWave_RefineCriterion; a neighbour
// that only exists on the coarser level counts as the cell itself), and by
// criterion 2 when rho exceeds the threshold.  Its flag buffer, the cube of
// 1 + 2 n_buffer cells around it, sets in its patch's mask the bit of every
// patch offset (dx,dy,dz) it reaches: (dz+1)*9 + (dy+1)*3 + (dx+1).
//
// Persistent blocks, each taking groups g = blockIdx.x, + gridDim.x, ...
// Per group the criterion's quantity of the group and of its one-cell halo
// is evaluated once per cell into shared memory, then every cell is tested.
// The next group's interior values, region table and halo values are
// loaded while the current group is tested, so that the block does not wait
// for memory between groups.
//
// The threshold comparisons run in T against thresholds rounded on the host
// so that they decide exactly as the comparison of the value widened to
// double with the double threshold: x >= d iff x >= (the least T >= d), and
// x > d iff x > (the greatest T <= d).  GB300's FP64 rate would otherwise
// make two FP64 operations per cell the largest cost of the kernel.
template <typename T, int CRIT>
__global__ void __launch_bounds__(NT_FLAG, (flag_blocks_per_sm<T, CRIT>()))
    k_flag(const FlagArgs<T> a, const T thr_ge, const T thr_gt) {
    constexpr int QC = CRIT == 1 ? 1 : 0;              // quantity: pressure or density
    constexpr bool HALO = CRIT != 2;
    constexpr int NFT = HALO ? 6 * GS * GS / NT_FLAG : 0;   // halo face cells per thread (3)
    using Q = SqPitch<T>;
    __shared__ T s_q[HP * Q::PLN];
    __shared__ int s_src[27], s_mask[27];
    __shared__ unsigned s_m[8];
    const int t = threadIdx.x;
    const size_t vs = (size_t)a.n_groups * 8 * 512;
    const T gm1 = T(a.gamma - 1.0);

    // Face cell k of the halo (the gradient criteria only; the edges and
    // corners of the halo are never read): its place in s_q, the group cell
    // next to it, and its value's source through the region table.  A face
    // cell whose region only exists on the coarser level takes the value of
    // that group cell, the one cell that reads it: the neighbour then counts
    // as the cell itself.
    auto face = [&](int k, int& idx, int& inner, size_t& off) -> bool {
        const int f = k >> 8, ax = f >> 1, a0 = k & 15, a1 = (k >> 4) & 15;
        const int e = (f & 1) ? GS : -1;                   // halo coordinate along ax
        int x = ax == 0 ? e : a0;
        int y = ax == 0 ? a0 : (ax == 1 ? e : a1);
        int z = ax == 2 ? e : a1;
        idx = Q::index(x, y, z);
        const int st = ax == 0 ? 1 : ax == 1 ? Q::RW : Q::PLN;
        inner = (f & 1) ? idx - st : idx + st;
        const int src = resolve(s_src, s_mask, x, y, z);
        off = src < 0 ? 0 : cell_offset(src, x, y, z);
        return src >= 0;
    };
    // the next group's interior (the group's own cells in memory order,
    // coalesced: local index j = ((patch * 8 + z) * 8 + y) * 8 + x with
    // patch = (pz * 2 + py) * 2 + px) and halo values, loaded ahead
    Raw<T, QC> nxt[PER_FLAG];
    Raw<T, QC> hnxt[NFT > 0 ? NFT : 1];
    bool hsame[NFT > 0 ? NFT : 1];
    // pass k covers patch k (x, y, z offsets 8 (k & 1), 8 ((k >> 1) & 1),
    // 8 (k >> 2)); within it the thread's cell is (t % 8, t / 8 % 8, t / 64)
    const int cx = t & 7, cy = (t >> 3) & 7, cz = t >> 6;
    const int tb = Q::index(cx, cy, cz);
    auto patch_off = [](int k) { return Q::index(8 * (k & 1), 8 * ((k >> 1) & 1), 8 * (k >> 2)) - Q::index(0, 0, 0); };
    // the patch offsets the flag buffer of this thread's cell reaches along
    // each axis, as 3-bit sets (bit d+1 for offset d), spread into the
    // 27-bit mask: the same for every patch of every group
    unsigned m_hit;
    {
        const int pc[3] = {cx, cy, cz};
        unsigned sa[3];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax)
            sa[ax] = 2u | (pc[ax] - a.n_buffer < 0 ? 1u : 0u) | (pc[ax] + a.n_buffer > PS - 1 ? 4u : 0u);
        const unsigned row = sa[0];
        const unsigned plane = ((sa[1] & 1u) ? row : 0u) | ((sa[1] & 2u) ? row << 3 : 0u) |
                               ((sa[1] & 4u) ? row << 6 : 0u);
        m_hit = ((sa[2] & 1u) ? plane : 0u) | ((sa[2] & 2u) ? plane << 9 : 0u) | ((sa[2] & 4u) ? plane << 18 : 0u);
    }
    int hidx[NFT > 0 ? NFT : 1], hinner[NFT > 0 ? NFT : 1];
    int g = blockIdx.x;
#pragma unroll
    for (int k = 0; k < PER_FLAG; ++k) nxt[k] = load_raw<T, QC>(a.u, vs, (size_t)g * CELLS_PG + k * NT_FLAG + t);
    if (HALO) {
        if (t < 27) region_entry(a.nbr, g, t, s_src, s_mask);
        __syncthreads();
#pragma unroll
        for (int i = 0; i < NFT; ++i) {
            size_t off;
            hsame[i] = face(i * NT_FLAG + t, hidx[i], hinner[i], off);
            if (hsame[i]) hnxt[i] = load_raw<T, QC>(a.u, vs, off);
        }
    }
    for (; g < a.n_groups; g += gridDim.x) {
        // the current group's interior and halo into shared memory
#pragma unroll
        for (int k = 0; k < PER_FLAG; ++k) s_q[tb + patch_off(k)] = quantity<T, QC>(nxt[k], gm1);
#pragma unroll
        for (int i = 0; i < NFT; ++i)
            if (hsame[i]) s_q[hidx[i]] = quantity<T, QC>(hnxt[i], gm1);
        if (t < 8) s_m[t] = 0u;
        __syncthreads();
        // coarse faces: the adjacent group cell, now in shared memory
#pragma unroll
        for (int i = 0; i < NFT; ++i)
            if (!hsame[i]) s_q[hidx[i]] = s_q[hinner[i]];
        // the next group's interior and region table
        const int gn = g + gridDim.x;
        const bool more = gn < a.n_groups;
        if (more) {
#pragma unroll
            for (int k = 0; k < PER_FLAG; ++k)
                nxt[k] = load_raw<T, QC>(a.u, vs, (size_t)gn * CELLS_PG + k * NT_FLAG + t);
            if (HALO && t < 27) region_entry(a.nbr, gn, t, s_src, s_mask);
        }
        __syncthreads();
        // the next group's halo: its region table is visible now, and the
        // loads are in flight during the tests below
        if (HALO && more) {
#pragma unroll
            for (int i = 0; i < NFT; ++i) {
                size_t off;
                hsame[i] = face(i * NT_FLAG + t, hidx[i], hinner[i], off);
                if (hsame[i]) hnxt[i] = load_raw<T, QC>(a.u, vs, off);
            }
        }
        // cells in memory order: pass k covers patch k, so the masks of a pass
        // combine by warp reductions before one shared atomic per warp
#pragma unroll
        for (int k = 0; k < PER_FLAG; ++k) {
            const int c0 = tb + patch_off(k);
            const T q0 = s_q[c0];
            bool hit;
            if (CRIT == 2) {
                hit = q0 > thr_gt;
            } else {
                // max over the axes of |q(+1) - q(-1)| / (2 |q|), ignoring NaN
                // ratios and starting from 0: the largest difference divided
                // once gives the same value, division by one denominator being
                // monotonic
                T n = fabs(s_q[c0 + 1] - s_q[c0 - 1]);
                n = fmax(n, fabs(s_q[c0 + Q::RW] - s_q[c0 - Q::RW]));
                n = fmax(n, fabs(s_q[c0 + Q::PLN] - s_q[c0 - Q::PLN]));
                const T r = n / (T(2) * fabs(q0));
                hit = (r > T(0) ? r : T(0)) >= thr_ge;
            }
            const unsigned m = __reduce_or_sync(0xffffffffu, hit ? m_hit : 0u);
            if ((t & 31) == 0 && m != 0u) atomicOr(&s_m[k], m);
        }
        __syncthreads();
        // the threads that reset s_m for the next group are the ones that
        // read it here; s_q is rewritten only after this barrier
        if (t < 8) a.masks[8 * g + t] = s_m[t];
    }
}

// The least T >= d and the greatest T <= d (NaN stays NaN, so that every
// comparison with it is false, as with d).
template <typename T>
static T round_up_to(double d) {
    if (sizeof(T) == sizeof(double)) return (T)d;
    const float f = (float)d;
    return (double)f < d ? nextafterf(f, INFINITY) : f;
}
template <typename T>
static T round_down_to(double d) {
    if (sizeof(T) == sizeof(double)) return (T)d;
    const float f = (float)d;
    return (double)f > d ? nextafterf(f, -INFINITY) : f;
}

template <typename T>
cudaError_t launch_flag(const FlagArgs<T>& a, cudaStream_t st) {
    if (a.n_groups <= 0) return cudaSuccess;
    const T ge = round_up_to<T>(a.threshold), gt = round_down_to<T>(a.threshold);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    auto grid = [&](int bps) { return a.n_groups < sms * bps ? a.n_groups : sms * bps; };
    if (a.criterion == 0) k_flag<T, 0><<<grid(flag_blocks_per_sm<T, 0>()), NT_FLAG, 0, st>>>(a, ge, gt);
    else if (a.criterion == 1) k_flag<T, 1><<<grid(flag_blocks_per_sm<T, 1>()), NT_FLAG, 0, st>>>(a, ge, gt);
    else k_flag<T, 2><<<grid(flag_blocks_per_sm<T, 2>()), NT_FLAG, 0, st>>>(a, ge, gt);
    return cudaGetLastError();
}
template cudaError_t launch_flag<float>(const FlagArgs<float>&, cudaStream_t);
template cudaError_t launch_flag<double>(const FlagArgs<double>&, cudaStream_t);

constexpr int NT_REF = 256;

// One block per group of the rebuilt level: a copy of the old group it
// inherits, or Min-Mod interpolation from its parent patch on the level
// below (the refinement step of Sec. 2.1).  Interpolation runs per coarse
// cell: a thread reads the cell and its six neighbours (through the coarse
// region table) once, forms the three limited slopes of each variable and
// writes all eight children, each as U + (sx Sx + sy Sy + sz Sz) / 4 in that
// order, the children of one x-pair as one paired store.
template <typename T>
__global__ void __launch_bounds__(NT_REF) k_refine(const RefineArgs<T> a) {
    __shared__ int s_csrc[27], s_cmask[27];
    const int g = blockIdx.x, t = threadIdx.x;
    const size_t vs = (size_t)a.n_new * 8 * 512;
    const int src = a.inherit[g];
    if (src >= 0) {
        // copy in chunks of VB variables, every load of a chunk issued before
        // its stores (all five variables at once in single precision)
        constexpr int N4 = CELLS_PG * (int)sizeof(T) / 16;
        constexpr int PER = N4 / NT_REF;
        constexpr int VB = sizeof(T) == 4 ? NV : 1;
        const size_t vso = (size_t)a.n_old * 8 * 512;
#pragma unroll 1
        for (int v0 = 0; v0 < NV; v0 += VB) {
            float4 buf[VB][PER];
#pragma unroll
            for (int v = 0; v < VB; ++v) {
                const float4* in =
                    reinterpret_cast<const float4*>(a.u_old + (v0 + v) * vso + (size_t)src * CELLS_PG);
#pragma unroll
                for (int i = 0; i < PER; ++i) buf[v][i] = __ldcs(in + i * NT_REF + t);
            }
#pragma unroll
            for (int v = 0; v < VB; ++v) {
                float4* out = reinterpret_cast<float4*>(a.u_new + (v0 + v) * vs + (size_t)g * CELLS_PG);
#pragma unroll
                for (int i = 0; i < PER; ++i) __stcs(out + i * NT_REF + t, buf[v][i]);
            }
        }
        return;
    }
    const int P = a.parent_new[g];
    if (t < 27) region_entry(a.nbrc, P >> 3, t, s_csrc, s_cmask);
    __syncthreads();
    const size_t vsc = (size_t)a.n_c * 8 * 512;
    const int px = P & 1, py = (P >> 1) & 1, pz = (P >> 2) & 1;
    constexpr int dd[7][3] = {{0, 0, 0}, {-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
#pragma unroll 1
    for (int i = t; i < PS * PS * PS; i += NT_REF) {
        // coarse cell (i % 8, i / 8 % 8, i / 64) of the parent patch
        const int ix = i & 7, iy = (i >> 3) & 7, iz = i >> 6;
        const int cx = PS * px + ix, cy = PS * py + iy, cz = PS * pz + iz;
        size_t off[7];
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            int xa = cx + dd[q][0], ya = cy + dd[q][1], za = cz + dd[q][2];
            const int s = resolve(s_csrc, s_cmask, xa, ya, za);
            off[q] = cell_offset(s < 0 ? 0 : s, xa, ya, za);   // s < 0 cannot pass host validation
        }
        T c[NV][7];
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
            for (int q = 0; q < 7; ++q) c[v][q] = a.uc[v * vsc + off[q]];
        // children (2 ix + dx, 2 iy + dy, 2 iz + dz) of the new group
        const size_t o0 = cell_offset(g, 2 * ix, 2 * iy, 2 * iz);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const T U = c[v][0];
            const T Sx = minmod_slope(c[v][1], U, c[v][2]);
            const T Sy = minmod_slope(c[v][3], U, c[v][4]);
            const T Sz = minmod_slope(c[v][5], U, c[v][6]);
#pragma unroll
            for (int dz = 0; dz < 2; ++dz)
#pragma unroll
                for (int dy = 0; dy < 2; ++dy) {
                    const T sy = dy ? T(1) : T(-1), sz = dz ? T(1) : T(-1);
                    const T lo = U + T(0.25) * ((T(-1) * Sx + sy * Sy) + sz * Sz);
                    const T hi = U + T(0.25) * ((T(1) * Sx + sy * Sy) + sz * Sz);
                    T* o = a.u_new + v * vs + o0 + dz * 64 + dy * 8;
                    if (sizeof(T) == 4) {
                        float2 w;
                        w.x = (float)lo;
                        w.y = (float)hi;
                        __stcs(reinterpret_cast<float2*>(o), w);
                    } else {
                        double2 w;
                        w.x = (double)lo;
                        w.y = (double)hi;
                        __stcs(reinterpret_cast<double2*>(o), w);
                    }
                }
        }
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
