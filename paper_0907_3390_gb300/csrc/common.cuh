// common.cuh -- device-side building blocks shared by the FP32 and FP64
// kernels: sizes, kernel argument structs, patch indexing, the ghost-zone
// gather (same-level copy, outflow clamp, Min-Mod interpolation from the
// coarser level) and the diagnostic helpers.
//
// Geometry (Sec. 3.1): a patch is 8^3 cells, a patch group the 2x2x2 oct of
// sibling patches (16^3 interior cells), padded by NG = 3 ghost cells per
// side for the seven-point stencil (Sec. 2.2) into a 22^3 block.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gh {

constexpr int NV = 5;      // rho, mx, my, mz, e
constexpr int PS = 8;      // patch size
constexpr int GS = 16;     // patch-group size
constexpr int NG = 3;      // ghost cells per side
constexpr int PD = 22;     // padded size
constexpr int MAXLEV = 16; // levels per launch
constexpr int CELLS_PG = GS * GS * GS;          // 4096
constexpr int FLUX_PG = 3 * 3 * NV * GS * GS;   // face-flux values per group
// Coarse-fine ghost slot of one FP32 group: per variable and padded x-row
// (zp, yp) 24 floats -- the 16 centre cells at 0..15, the -x edge (x = -3..-1)
// at 16..18, the +x edge (x = 16..18) at 20..22 -- so every piece starts on
// a 16-byte boundary.
constexpr int GROW = 24;
constexpr int GVS = PD * PD * GROW;             // floats per variable of a slot
constexpr size_t GHOST_PG = (size_t)NV * GVS;   // floats per slot

// One level as a kernel sees it.  All pointers are device memory.
template <typename T>
struct LevelArgs {
    const T* u;         // [5][8n][8][8][8] pre-step state
    T* u_out;           // post-step state
    const int* nbr;     // [n][26]
    T* flux;            // [n][3][3][5][16][16] or nullptr
    const int* parent;  // [n] patch index on level-1, nullptr on level 0
    const T* uc;        // level-1 pre-step state (coarse ghosts)
    const T* ucn;       // level-1 state after its sweep set (individual time steps), or nullptr
    const int* nbrc;    // level-1 map
    T* ghost;           // FP32: the coarse-fine ghost cells of this launch, formed by a pass before the
                        // sweeps ([slot][5][22][22][24]), or nullptr (level 0, FP64)
    const int* gslot;   // [n] slot of a group in ghost, -1 for a group with no coarse region
    const int* slot_g;  // [n_slots] group of each slot
    int n_groups;
    int n_groups_c;
    int item0;          // first work item of this level in a multi-level launch
    int n_slots;
    double dh;          // cell width; lambda = dt * dts / dh is formed on the device in FP64
    double dts;         // this level's share of the device dt: 1, or 2^-l with individual time steps
    double cw;          // time weight of ucn in the coarse ghosts (0 or 1/2)
    const unsigned* fneed;  // FP32, handle-owned fluxes: [n] bit 4 ax + q set where the fix-ups read a
                            // flux of the axis-ax sweep columns in transverse quarter q; nullptr: all
};

// Per-group diagnostic sinks (exact max of the signal speed, leaf sums of
// the conserved variables, count of bad leaf cells), indexed by work item.
struct DiagSink {
    unsigned long long* pg_max;
    double* pg_sum;     // [item][5]
    int* pg_bad;
};

struct StepOut;

// End-of-step reduction run by the CTA that finishes last in a
// single-level launch with fused diagnostics; out == nullptr turns it off.
struct StepSink {
    StepOut* out;       // device copy of the result
    StepOut* out_host;  // mapped pinned host copy, or nullptr
    double* dt;         // the launch's dt slot, rewritten after every item is done
    double cfl;
    double dh;
    int update_dt;
    int n_items;        // per-group diagnostic entries to combine
};

// An xyz set followed by a zyx set of one level in one launch (same dt).
// Work items [0, n) are the xyz set of group i (u -> u_out); items [n, 2n)
// the zyx set of group order1[i - n] (u_out -> u), which starts once the
// xyz results of that group and of its 26 neighbours are published:
// ready[g] == *epoch + 1.  ready == nullptr turns it off.
struct PairArgs {
    unsigned* ready;    // [n] per-group publication marks
    unsigned* epoch;    // launch counter; the last CTA advances it
    unsigned* status;   // nonzero after a wait gave up (reported, then cleared)
    const int* order1;  // [n] zyx work order
    int hold;           // a group whose xyz mark is not published (the failure-path test), or -1
};

template <typename T>
struct SweepArgs {
    LevelArgs<T> lv[MAXLEV];
    int n_levels;
    int total;          // work items (patch groups) over all levels
    int* queue;         // device work-queue counter, zero before launch
    unsigned* done;     // count of CTAs that finished, zero before launch; the
                        // last CTA sets both back to zero
    const double* dt;   // device slot holding the time step
    DiagSink diag;      // fused diagnostics of the new state, or all null
    StepSink step;      // fused end-of-step reduction (needs diag), or all null
    PairArgs pair;      // xyz + zyx pair launch, or all null
    T gamma;
    T gm1;              // gamma - 1, formed once on the host in FP64
};

__host__ __device__ __forceinline__ int dir_index(int dx, int dy, int dz) {
    int d = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
    return d < 13 ? d : d - 1;
}

// Offset of cell (x,y,z), 0 <= x,y,z < 16, of group g inside one variable's
// array of the patch layout.
__device__ __forceinline__ size_t cell_offset(int g, int x, int y, int z) {
    int patch = (((z >> 3) << 1 | (y >> 3)) << 1) | (x >> 3);
    return ((size_t)(8 * g + patch) << 9) + (size_t)((((z & 7) << 3) | (y & 7)) << 3 | (x & 7));
}

// Region table of one group: for each of the 27 regions r = (oz+1)*9 +
// (oy+1)*3 + (ox+1) around it, the source group after outflow clamping
// (axes whose face neighbour is -2 are clamped into the group first), and
// the clamp mask (bit a set = clamp axis a).  src = -1: coarse region.
// Called by 27 threads.
__device__ __forceinline__ void region_entry(const int* __restrict__ nbr, int g, int r,
                                             int* s_src, int* s_mask) {
    int o[3] = {r % 3 - 1, (r / 3) % 3 - 1, r / 9 - 1};
    int mask = 0;
    for (int a = 0; a < 3; ++a) {
        if (o[a] != 0) {
            int e[3] = {0, 0, 0};
            e[a] = o[a];
            if (nbr[(size_t)g * 26 + dir_index(e[0], e[1], e[2])] == -2) {
                mask |= 1 << a;
                o[a] = 0;
            }
        }
    }
    int src = g;
    if (o[0] | o[1] | o[2]) src = nbr[(size_t)g * 26 + dir_index(o[0], o[1], o[2])];
    s_src[r] = src;
    s_mask[r] = mask;
}

__device__ __forceinline__ int region_of(int c) { return c < 0 ? -1 : (c >= GS ? 1 : 0); }

// Resolve a group-local position (-16 <= c < 32) through a region table:
// returns the source group (or -1 / < -1) and rewrites c into it.
__device__ __forceinline__ int resolve(const int* s_src, const int* s_mask, int& x, int& y, int& z) {
    int ox = region_of(x), oy = region_of(y), oz = region_of(z);
    int r = (oz + 1) * 9 + (oy + 1) * 3 + (ox + 1);
    int m = s_mask[r];
    x = (m & 1) ? min(max(x, 0), GS - 1) : x - GS * ox;
    y = (m & 2) ? min(max(y, 0), GS - 1) : y - GS * oy;
    z = (m & 4) ? min(max(z, 0), GS - 1) : z - GS * oz;
    return s_src[r];
}

template <typename T>
__device__ __forceinline__ T minmod_slope(T l, T c, T r) {
    T a = c - l, b = r - c;
    if (a * b > T(0)) {
        T m = fmin(fabs(a), fabs(b));
        return a > T(0) ? m : -m;
    }
    return T(0);
}

// Conservative linear interpolation with the Min-Mod limiter (Sec. 2.1
// refinement step, Sec. 2.2 ghost zones) of the fine ghost cell at
// group-local (x,y,z) of a group whose parent patch has local position
// (px,py,pz) in coarse group gc.  Coarse data: the coarse level's pre-step
// state uc, resolved through the coarse region table.  Writes NV values.
template <typename T>
__device__ __forceinline__ void prolong(const T* __restrict__ uc, const T* __restrict__ ucn, T w,
                                        size_t vstride_c, const int* s_csrc, const int* s_cmask, int px,
                                        int py, int pz, int x, int y, int z, T out[NV]) {
    const int cx = PS * px + (x >> 1), cy = PS * py + (y >> 1), cz = PS * pz + (z >> 1);
    const T sx = (x & 1) ? T(1) : T(-1);
    const T sy = (y & 1) ? T(1) : T(-1);
    const T sz = (z & 1) ? T(1) : T(-1);
    size_t off[7];
    const int dd[7][3] = {{0, 0, 0}, {-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        int a = cx + dd[q][0], b = cy + dd[q][1], c = cz + dd[q][2];
        int s = resolve(s_csrc, s_cmask, a, b, c);
        off[q] = cell_offset(s < 0 ? 0 : s, a, b, c);   // s < 0 cannot pass host validation
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const T* p = uc + v * vstride_c;
        T c[7];
#pragma unroll
        for (int q = 0; q < 7; ++q) c[q] = p[off[q]];
        if (ucn != nullptr) {
            // individual time steps: the coarse state at the start of this
            // level's step, linear in time between before and after the
            // coarse sweep set
            const T* pn = ucn + v * vstride_c;
#pragma unroll
            for (int q = 0; q < 7; ++q) c[q] = c[q] + w * (pn[off[q]] - c[q]);
        }
        T U = c[0];
        T Sx = minmod_slope(c[1], U, c[2]);
        T Sy = minmod_slope(c[3], U, c[4]);
        T Sz = minmod_slope(c[5], U, c[6]);
        T t = (sx * Sx + sy * Sy) + sz * Sz;
        out[v] = U + T(0.25) * t;
    }
}

// Fill the padded block blk (pitches XP along x, PD rows along y, PD
// planes along z, VS per variable) of group g on level L by all threads of
// the block.  s_src/s_mask: region table of g; s_csrc/s_cmask: region table
// of the parent's coarse group (only read where a region is -1).
template <typename T, int XP, int NT>
__device__ __forceinline__ void gather_block(T* blk, size_t VS, const LevelArgs<T>& L, int g,
                                             const int* s_src, const int* s_mask,
                                             const int* s_csrc, const int* s_cmask, int ppx,
                                             int ppy, int ppz) {
    const size_t vstride = (size_t)L.n_groups * 8 * 512;
    const size_t vstride_c = (size_t)L.n_groups_c * 8 * 512;
    for (int i = threadIdx.x; i < PD * PD * PD; i += NT) {
        int xp = i % PD, t = i / PD;
        int yp = t % PD, zp = t / PD;
        int x = xp - NG, y = yp - NG, z = zp - NG;
        int s = resolve(s_src, s_mask, x, y, z);
        T* d = blk + ((size_t)zp * PD + yp) * XP + xp;
        if (s >= 0) {
            const T* p = L.u + cell_offset(s, x, y, z);
#pragma unroll
            for (int v = 0; v < NV; ++v) d[v * VS] = p[v * vstride];
        } else {
            T val[NV];
            prolong<T>(L.uc, L.ucn, (T)L.cw, vstride_c, s_csrc, s_cmask, ppx, ppy, ppz, xp - NG, yp - NG, zp - NG,
                       val);
#pragma unroll
            for (int v = 0; v < NV; ++v) d[v * VS] = val[v];
        }
    }
}

// Build the region tables of group g (and of its parent's coarse group when
// the level has a parent map).  Threads 0..26 and 32..58 of the block.
template <typename T>
__device__ __forceinline__ void build_tables(const LevelArgs<T>& L, int g, int* s_src, int* s_mask,
                                             int* s_csrc, int* s_cmask, int* s_par) {
    int t = threadIdx.x;
    if (t < 27) region_entry(L.nbr, g, t, s_src, s_mask);
    if (L.parent != nullptr) {
        int P = L.parent[g];
        if (t >= 32 && t < 59) region_entry(L.nbrc, P >> 3, t - 32, s_csrc, s_cmask);
        if (t == 0) s_par[0] = P;
    } else if (t == 0) {
        s_par[0] = -1;
    }
}

// FP32 signal speed c_s + max(|vx|,|vy|,|vz|) (denominator of Eq. CFL) and
// pressure (Eqs. ThermalEnergy, EOS), written with explicitly rounded
// intrinsics so that every translation unit evaluates it identically
// whatever its contraction and precision flags.
__device__ __forceinline__ void speed_pressure_f32(const float u[NV], float g, float gm1, float& s,
                                                   float& P) {
    const float ri = __fdividef(1.0f, u[0]);
    const float m2 = fmaf(u[1], u[1], fmaf(u[2], u[2], __fmul_rn(u[3], u[3])));
    P = __fmul_rn(gm1, fmaf(__fmul_rn(-0.5f, ri), m2, u[4]));
    const float x = __fmul_rn(__fmul_rn(g, fmaxf(P, 0.0f)), ri);
    // sqrt(x) through the reciprocal square root; x = 0 gives 0, a negative
    // or NaN x gives NaN (as sqrt would)
    const float cs = x == 0.0f ? 0.0f : __fmul_rn(x, rsqrtf(x));
    s = fmaf(fmaxf(fmaxf(fabsf(u[1]), fabsf(u[2])), fabsf(u[3])), ri, cs);
}

// Exact-order maximum of positive doubles through their bit patterns.
__device__ __forceinline__ void atomic_max_pos(unsigned long long* addr, double v) {
    atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

}  // namespace gh
