// sweep_f32.cu -- batched FP32 relaxing-TVD patch-group kernel.
//
// One persistent launch advances the patch groups of every level by one
// sweep set (Sec. 3.1).  Each CTA owns one SM (the padded block fills
// shared memory) and pulls work items -- (level, group) pairs -- from a
// device counter with atomicAdd.  For each item it
//   1. gathers the padded 22^3 x 5 block into shared memory: interior and
//      same-level ghosts copied, outflow faces clamped, coarse ghosts
//      interpolated with the Min-Mod limiter from the coarser level
//      (Sec. 2.2, Sec. 3.1);
//   2. runs the three directional sweeps (xyz or zyx, Sec. 2.2) on chip.
//      A thread owns a whole 1-D column and streams along it with a
//      register window, so the half step (Eq. MidpointValue), the TVD
//      fluxes (Eqs. 2ndTVDFluxCorr..2ndRFlux) and the full step
//      (Eq. FullstepValue) never leave registers; results overwrite the
//      column in place.  The x sweep updates 16 cells of 22x22 columns, y
//      16 of 16x22, z 16 of 16x16 (the shrinking regions of the 7-point
//      stencil);
//   3. writes the 16^3 interior to u_out (and the face fluxes on planes 0,
//      8, 16 of each axis when a flux buffer is given).
//
// Arithmetic: with A = c u + F = 2 F^R and B = c u - F = 2 F^L (Eq.
// LRFlux, w = F/c substituted), the upwind interface flux of the half step
// is (A_n - B_{n+1})/2, and the TVD fluxes are
//   A_{n+1/2} = A_n     + psi(A_n - A_{n-1}, A_{n+1} - A_n),
//   B_{n+1/2} = B_{n+1} - psi(B_{n+2} - B_{n+1}, B_{n+1} - B_n),
// where psi(x, y) = phi(x/4, y/4) * 2 by homogeneity of the limiter:
// van Leer gives xy/(x+y) when xy > 0, minmod gives min(|x|,|y|)/2 with
// the common sign.  All factors of 2 are exact.  Reciprocal, division and
// square root use the fast single-precision forms (this file is compiled
// with -prec-div=false -prec-sqrt=false -ftz=true).
#include "common.cuh"
#include "internal.h"
#include "lane_maps.h"

namespace gh {

constexpr int XP = 23;                    // x pitch: odd, so x-sweep columns hit distinct banks
constexpr int VS = PD * PD * XP;          // floats per variable in shared memory
constexpr size_t SMEM_F32 = (size_t)NV * VS * sizeof(float) + 512 * sizeof(int);   // block + item tables + counters + reduction

// A = c u + F (= 2 F^R) and B = c u - F (= 2 F^L) of one cell for a sweep
// along AXIS (Eq. LRFlux with w = F/c substituted): c = |v_n| + c_s
// (Sec. 2.2), F = (m_n, m v_n + P e_n, (e + P) v_n), P from Eqs.
// ThermalEnergy, EOS.
template <int AXIS>
__device__ __forceinline__ void state(const float u[NV], float g, float gm1, float A[NV], float B[NV]) {
    const float r = u[0];
    const float ri = __fdividef(1.0f, r);
    const float mn = u[1 + AXIS];
    const float vn = mn * ri;
    const float m2 = fmaf(u[1], u[1], fmaf(u[2], u[2], u[3] * u[3]));
    const float P = gm1 * fmaf(-0.5f * ri, m2, u[4]);
    const float cs = sqrtf(g * fmaxf(P, 0.0f) * ri);
    const float c = fabsf(vn) + cs;
    float F[NV];
    F[0] = mn;
    F[1] = u[1] * vn;
    F[2] = u[2] * vn;
    F[3] = u[3] * vn;
    F[1 + AXIS] = fmaf(mn, vn, P);
    F[4] = (u[4] + P) * vn;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        A[v] = fmaf(c, u[v], F[v]);
        B[v] = fmaf(c, u[v], -F[v]);
    }
}

// base + s psi(x, y), s = +1 or -1, with psi(x, y) = 2 phi(x/4, y/4): by
// homogeneity of the limiter, on unhalved differences of A or B.  van Leer
// (Eq. vanLeer): xy/(x+y) when xy > 0, here as one FMA of xy with
// s/(x+y); minmod: min(|x|,|y|)/2 with the common sign; zero otherwise.
template <int LIM>
__device__ __forceinline__ float add_psi(float base, float x, float y, float s) {
    const float p = x * y;
    if (LIM == 0) {
        const float r = __fdividef(s, x + y);
        return p > 0.0f ? fmaf(p, r, base) : base;
    } else {
        const float m = 0.5f * fminf(fabsf(x), fabsf(y));
        return p > 0.0f ? base + s * copysignf(m, x) : base;
    }
}

// Register state carried along one column.
struct ColState {
    float u1[NV];          // u_{k-1}
    float Ap[NV];          // A_{k-1}
    float Hp[NV];          // half-step flux (x2) at interface k-3/2
    float Aq[NV], Bq[NV];  // A', B' of the midpoint state of cell k-2
    float dAp[NV], dBp[NV];// dA', dB' at interface k-5/2
    float Ahp[NV];         // TVD A' flux at interface k-5/2
    float Gp[NV];          // net flux (x2) at interface k-7/2
};

// Step k of the stream along a column.  K = min(k, 6) is the fill level of
// the pipeline (compile time): cell k enters (K >= 0); the half-step flux
// at k-1/2 forms (K >= 1, Eq. MidpointValue with first-order upwind
// fluxes); the midpoint state of cell k-1 and its A', B' form (K >= 2);
// the differences at k-3/2 (K >= 3); the TVD fluxes A'_{k-3/2} and
// B'_{k-5/2} (K >= 4, Eqs. 2ndTVDFluxCorr..2ndRFlux and their left-moving
// mirror); the net flux at k-5/2 (K >= 5); the full step of cell k-3
// (K >= 6, Eq. FullstepValue).
template <int AXIS, int S, int LIM, int K>
__device__ __forceinline__ void col_step(float* __restrict__ p, int k, ColState& c, float lam4,
                                         float lam2, float g, float gm1, float* __restrict__ fl) {
    float u[NV], A[NV], B[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) u[v] = p[k * S + v * VS];
    state<AXIS>(u, g, gm1, A, B);
    if (K >= 1) {
        float H[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) H[v] = c.Ap[v] - B[v];
        if (K >= 2) {
            float uh[NV], A1[NV], B1[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) uh[v] = fmaf(-lam4, H[v] - c.Hp[v], c.u1[v]);
            state<AXIS>(uh, g, gm1, A1, B1);
            if (K >= 3) {
                float dA[NV], dB[NV];
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    dA[v] = A1[v] - c.Aq[v];
                    dB[v] = B1[v] - c.Bq[v];
                }
                if (K >= 4) {
                    float G[NV];
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        const float Ah = add_psi<LIM>(c.Aq[v], c.dAp[v], dA[v], 1.0f);
                        const float Bh = add_psi<LIM>(c.Bq[v], dB[v], c.dBp[v], -1.0f);
                        G[v] = c.Ahp[v] - Bh;                    // net flux (x2) at k-5/2
                        c.Ahp[v] = Ah;
                    }
                    if (K >= 5) {
                        if (fl != nullptr && ((k - 5) & 7) == 0) {
#pragma unroll
                            for (int v = 0; v < NV; ++v) fl[((k - 5) >> 3) * (NV * 256) + v * 256] = 0.5f * G[v];
                        }
                        if (K >= 6) {
#pragma unroll
                            for (int v = 0; v < NV; ++v) {
                                const float un = p[(k - 3) * S + v * VS];
                                p[(k - 3) * S + v * VS] = fmaf(-lam2, G[v] - c.Gp[v], un);
                            }
                        }
#pragma unroll
                        for (int v = 0; v < NV; ++v) c.Gp[v] = G[v];
                    }
                }
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    c.dAp[v] = dA[v];
                    c.dBp[v] = dB[v];
                }
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                c.Aq[v] = A1[v];
                c.Bq[v] = B1[v];
            }
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) c.Hp[v] = H[v];
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        c.Ap[v] = A[v];
        c.u1[v] = u[v];
    }
}

// One 1-D column of 22 cells starting at p (stride S between cells, VS
// between variables) along AXIS; cells 3..18 are overwritten with the
// full-step values.  fl: face-flux slot of this row ([3 planes][5][256]
// with plane stride 5*256), or nullptr.  Cells 0..5 fill the pipeline
// (unrolled), cells 6..21 run the rolled steady-state step, which keeps the
// code small enough for the instruction cache.
template <int AXIS, int S, int LIM>
__device__ __forceinline__ void column(float* __restrict__ p, float lam4, float lam2, float g,
                                       float gm1, float* __restrict__ fl) {
    ColState c;
    col_step<AXIS, S, LIM, 0>(p, 0, c, lam4, lam2, g, gm1, fl);
    col_step<AXIS, S, LIM, 1>(p, 1, c, lam4, lam2, g, gm1, fl);
    col_step<AXIS, S, LIM, 2>(p, 2, c, lam4, lam2, g, gm1, fl);
    col_step<AXIS, S, LIM, 3>(p, 3, c, lam4, lam2, g, gm1, fl);
    col_step<AXIS, S, LIM, 4>(p, 4, c, lam4, lam2, g, gm1, fl);
    col_step<AXIS, S, LIM, 5>(p, 5, c, lam4, lam2, g, gm1, fl);
#pragma unroll 2
    for (int k = 6; k < PD; ++k) col_step<AXIS, S, LIM, 6>(p, k, c, lam4, lam2, g, gm1, fl);
}

// Column order of sweep S_IDX of an ORDER set that avoids shared-memory
// bank conflicts within a warp (lane_maps.h), or nullptr where the natural
// order is kept.
template <int ORDER, int S_IDX>
__device__ __forceinline__ const unsigned short* lane_map() {
    if (ORDER == 0) return S_IDX == 1 ? kLaneXyzS2 : nullptr;
    return S_IDX == 0 ? kLaneZyxS1 : S_IDX == 1 ? kLaneZyxS2 : kLaneZyxS3;
}

// Face-flux slot of the column at transverse position (i1, i2) of a sweep
// along AX, or nullptr where the group has no flux buffer, the column is
// not an interior one, or (MASK) no fix-up reads its fluxes (fm: bit 4 AX +
// q for the transverse quarter q = 2 [(i2 - 3) >= 8] + [(i1 - 3) >= 8]).
template <int AX, bool MASK>
__device__ __forceinline__ float* flux_slot(float* flux_g, unsigned fm, int i1, int i2) {
    float* fl = nullptr;
    if (flux_g != nullptr && i1 >= NG && i1 < NG + GS && i2 >= NG && i2 < NG + GS &&
        (!MASK || ((fm >> (4 * AX + 2 * ((i2 - NG) >> 3) + ((i1 - NG) >> 3))) & 1u)))
        fl = flux_g + AX * (3 * NV * 256) + (i2 - NG) * GS + (i1 - NG);
    return fl;
}

// Sweep s (0,1,2) of order ORDER over the shared block; columns whose
// transverse axes were swept earlier in this set only cover [3,19).
template <int ORDER, int S_IDX, int LIM, bool MASK = false>
__device__ __forceinline__ void sweep(float* sm, float lam, float g, float gm1, float* flux_g, int nact,
                                      unsigned fm = 0xFFFu) {
    constexpr int AX = ORDER == 0 ? S_IDX : 2 - S_IDX;
    constexpr int T1 = AX == 0 ? 1 : 0;
    constexpr int T2 = AX == 2 ? 1 : 2;
    // axis done before this sweep?
    constexpr bool D1 = ORDER == 0 ? (T1 < AX) : (T1 > AX);
    constexpr bool D2 = ORDER == 0 ? (T2 < AX) : (T2 > AX);
    constexpr int LO1 = D1 ? NG : 0, N1 = D1 ? GS : PD;
    constexpr int LO2 = D2 ? NG : 0, N2 = D2 ? GS : PD;
    constexpr int ST[3] = {1, XP, PD * XP};
    constexpr int S = ST[AX];
    const float lam4 = 0.25f * lam, lam2 = 0.5f * lam;
    if ((int)threadIdx.x >= nact) return;
    const unsigned short* map = lane_map<ORDER, S_IDX>();
    for (int c = threadIdx.x; c < N1 * N2; c += nact) {
        int i1, i2;
        if (map != nullptr) {
            const unsigned m = __ldg(map + c);
            i1 = m & 255u;
            i2 = m >> 8;
        } else {
            i1 = LO1 + c % N1;
            i2 = LO2 + c / N1;
        }
        float* p = sm + i1 * ST[T1] + i2 * ST[T2];
        column<AX, S, LIM>(p, lam4, lam2, g, gm1, flux_slot<AX, MASK>(flux_g, fm, i1, i2));
    }
}

// ---------------------------------------------------------------- gather

__device__ __forceinline__ float4 ldg4(const float* p) {
    return __ldg(reinterpret_cast<const float4*>(p));
}

__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Work-item context in shared memory: region tables of the group and of its
// parent's coarse group, level, group index and parent patch.
struct ItemTab {
    int src[27], mask[27], csrc[27], cmask[27];
    int item, level, g, par, gslot;
    float lam;          // dt / dh, formed in FP64 from the device time step
};

__device__ __forceinline__ int level_of(const SweepArgs<float>& a, int item) {
    int l = 0;
    while (l + 1 < a.n_levels && item >= a.lv[l + 1].item0) ++l;
    return l;
}

// Threads t0..t0+26 and t0+32..t0+58 of the block.
__device__ __forceinline__ void build_tab(ItemTab& t, const SweepArgs<float>& a, int item, int t0) {
    const int l = level_of(a, item);
    const LevelArgs<float>& L = a.lv[l];
    int g = item - L.item0;
    if (a.pair.ready != nullptr && l == 1) g = a.pair.order1[g];   // zyx half of a pair launch
    const int tid = (int)threadIdx.x - t0;
    if (tid >= 0 && tid < 27) region_entry(L.nbr, g, tid, t.src, t.mask);
    if (tid >= 32 && tid < 59 && L.parent != nullptr)
        region_entry(L.nbrc, L.parent[g] >> 3, tid - 32, t.csrc, t.cmask);
    if (tid == 0) {
        t.item = item;
        t.level = l;
        t.g = g;
        t.par = L.parent != nullptr ? L.parent[g] : -1;
        t.gslot = L.gslot != nullptr ? L.gslot[g] : -1;
        t.lam = (float)((*a.dt * L.dts) / L.dh);
    }
}

// The interior of a work item into L2 (5 contiguous 16 KiB runs).
__device__ __forceinline__ void prefetch_item(const SweepArgs<float>& a, int item) {
    const int l = level_of(a, item);
    const LevelArgs<float>& L = a.lv[l];
    int g = item - L.item0;
    if (a.pair.ready != nullptr && l == 1) g = a.pair.order1[g];
    const size_t vs = (size_t)L.n_groups * 8 * 512;
    const float* b = L.u + ((size_t)g << 12);
#pragma unroll
    for (int v = 0; v < NV; ++v) prefetch_l2(b + v * vs, CELLS_PG * sizeof(float));
}

// Coarse-fine ghost cell by Min-Mod interpolation.  Kept out of line: it is
// the cold path of the gathers (coarse-fine faces only), and inlining it at
// every gather site made the kernel's code large enough to miss in the
// instruction cache on the hot path.
__device__ __noinline__ void prolong_cell(const LevelArgs<float>& L, const ItemTab& t, int x, int y,
                                             int z, float val[NV]) {
    const int lp = t.par & 7;
    prolong<float>(L.uc, L.ucn, (float)L.cw, (size_t)L.n_groups_c * 8 * 512, t.csrc, t.cmask, lp & 1, (lp >> 1) & 1,
                   (lp >> 2) & 1, x, y, z, val);
}

// One padded x-row (yp, zp) of the block of item t.  SEG bit 0: the 16
// centre cells (x in [0,16)); bit 1: the 3 + 3 edge cells; bit 2 / bit 3:
// only the first / second half of the centre (one patch row each).  Every cell lies
// in an aligned quad of a patch row of its source group, so the centre is
// four 16-byte loads per variable and each edge one.  Outflow edges repeat
// the centre's edge cell (zero gradient).  Cells of coarse regions are read
// from the group's ghost slot in ROWI launches (one 16-byte load per
// piece, like a same-level row) and interpolated one by one otherwise.
template <int SEG, bool ROWI = false>
__device__ __forceinline__ void gather_row(float* sm, const SweepArgs<float>& a, const ItemTab& t,
                                           int yp, int zp) {
    const LevelArgs<float>& L = a.lv[t.level];
    const size_t vstride = (size_t)L.n_groups * 8 * 512;
    float* d = sm + (zp * PD + yp) * XP;
    const int y = yp - NG, z = zp - NG;
    int xc = 0, yc = y, zc = z;
    const int sc = resolve(t.src, t.mask, xc, yc, zc);
    const size_t offc = sc >= 0 ? cell_offset(sc, 0, yc, zc) : 0;
    constexpr bool H0 = (SEG & 1) || (SEG & 4), H1 = (SEG & 1) || (SEG & 8);
    // ROWI: the launch's coarse-fine ghost cells were formed before it, in
    // the group's ghost slot (k_ghost_f32)
    const float* gp = ROWI && t.gslot >= 0 ? L.ghost + (size_t)t.gslot * GHOST_PG + (zp * PD + yp) * GROW : nullptr;
    if (H0 || H1) {
        if (sc >= 0 || ROWI) {
            // the row's centre from its group (patch px = 1 at +512) or from
            // the ghost slot (x = 8 at +8)
            const float* p0 = sc >= 0 ? L.u + offc : gp;
            const size_t vst = sc >= 0 ? vstride : (size_t)GVS;
            const int o1 = sc >= 0 ? 512 : PS;
            float4 c[NV][4];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const float* p = p0 + v * vst;
                if (H0) {
                    c[v][0] = ldg4(p);
                    c[v][1] = ldg4(p + 4);
                }
                if (H1) {
                    c[v][2] = ldg4(p + o1);
                    c[v][3] = ldg4(p + o1 + 4);
                }
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                float* q = d + v * VS + NG;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if ((j < 2 && !H0) || (j >= 2 && !H1)) continue;
                    q[4 * j + 0] = c[v][j].x;
                    q[4 * j + 1] = c[v][j].y;
                    q[4 * j + 2] = c[v][j].z;
                    q[4 * j + 3] = c[v][j].w;
                }
            }
        } else {
            for (int x = H0 ? 0 : PS; x < (H1 ? GS : PS); ++x) {
                float val[NV];
                prolong_cell(L, t, x, y, z, val);
#pragma unroll
                for (int v = 0; v < NV; ++v) d[v * VS + NG + x] = val[v];
            }
        }
    }
    if (SEG & 2) {
        const int rb = (region_of(z) + 1) * 9 + (region_of(y) + 1) * 3;
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const int o = side == 0 ? 0 : NG + GS;       // first padded cell of the edge
            if (t.mask[rb + 2 * side] & 1) {
                // outflow along x: the centre's cell at x = 0 or 15, three times
                float val[NV];
                if (sc >= 0) {
#pragma unroll
                    for (int v = 0; v < NV; ++v) val[v] = L.u[v * vstride + offc + (side ? 512 + 7 : 0)];
                } else if (ROWI) {
#pragma unroll
                    for (int v = 0; v < NV; ++v) val[v] = gp[v * GVS + (side ? GS - 1 : 0)];
                } else {
                    prolong_cell(L, t, side ? GS - 1 : 0, y, z, val);
                }
#pragma unroll
                for (int v = 0; v < NV; ++v) d[v * VS + o] = d[v * VS + o + 1] = d[v * VS + o + 2] = val[v];
                continue;
            }
            int xs = side ? GS : -1, ys = y, zs = z;
            const int se = resolve(t.src, t.mask, xs, ys, zs);
            if (se >= 0) {
                // x = 12..15 of the -x neighbour's px = 1 row, or x = 0..3 of the +x one
                const size_t off = cell_offset(se, 0, ys, zs) + (side ? 0 : 512 + 4);
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const float4 q = ldg4(L.u + v * vstride + off);
                    if (side == 0) {
                        d[v * VS + 0] = q.y;
                        d[v * VS + 1] = q.z;
                        d[v * VS + 2] = q.w;
                    } else {
                        d[v * VS + 19] = q.x;
                        d[v * VS + 20] = q.y;
                        d[v * VS + 21] = q.z;
                    }
                }
            } else if (ROWI) {
                // x = -3..-1 at 16, x = 16..18 at 20
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const float4 q = ldg4(gp + v * GVS + (side ? 20 : 16));
                    d[v * VS + o] = q.x;
                    d[v * VS + o + 1] = q.y;
                    d[v * VS + o + 2] = q.z;
                }
            } else {
                for (int k = 0; k < NG; ++k) {
                    float val[NV];
                    prolong_cell(L, t, side ? GS + k : k - NG, y, z, val);
#pragma unroll
                    for (int v = 0; v < NV; ++v) d[v * VS + o + k] = val[v];
                }
            }
        }
    }
}

// Row sets of the pipelined gather of the next item, chosen so that each
// set only writes cells the current item no longer reads:
//   xyz: A during sweep 2: x-edges of all rows; B during sweep 3: centres of
//        rows outside [3,19) in y; C during the store: centres of rows
//        outside [3,19) in z (inside in y); D after the store: centres of
//        the 16x16 interior rows.
//   zyx: A: full rows outside [3,19) in z; B: full rows inside in z,
//        outside in y; C: x-edges of the interior rows; D: their centres.
__device__ __forceinline__ int ghost_row(int q) { return q < NG ? q : q + GS; }   // 0..5 -> 0,1,2,19,20,21

template <int ORDER, int PH>
struct GatherSet {
    static constexpr int N = ORDER == 0 ? (PH == 0 ? PD * PD : PH == 1 ? 6 * PD : PH == 2 ? 6 * GS : 2 * GS * GS)
                                        : (PH == 0 ? 6 * PD : PH == 1 ? 6 * GS : PH == 2 ? GS * GS : 2 * GS * GS);
};

// Task r of set PH (set D is split into half rows so that every thread
// gets one).
template <int ORDER, int PH, bool ROWI = false>
__device__ __forceinline__ void gather_task(float* sm, const SweepArgs<float>& a, const ItemTab& t, int r) {
    if (PH == 3) {
        const int row = r >> 1;
        if (r & 1) gather_row<8, ROWI>(sm, a, t, NG + row % GS, NG + row / GS);
        else gather_row<4, ROWI>(sm, a, t, NG + row % GS, NG + row / GS);
        return;
    }
    int yp, zp;
    if (ORDER == 0) {
        if (PH == 0) { yp = r % PD; zp = r / PD; }
        else if (PH == 1) { yp = ghost_row(r % 6); zp = r / 6; }
        else { yp = NG + r % GS; zp = ghost_row(r / GS); }
        if (PH == 0) gather_row<2, ROWI>(sm, a, t, yp, zp);
        else gather_row<1, ROWI>(sm, a, t, yp, zp);
    } else {
        if (PH == 0) { yp = r % PD; zp = ghost_row(r / PD); }
        else if (PH == 1) { yp = ghost_row(r % 6); zp = NG + r / 6; }
        else { yp = NG + r % GS; zp = NG + r / GS; }
        if (PH <= 1) gather_row<3, ROWI>(sm, a, t, yp, zp);
        else gather_row<2, ROWI>(sm, a, t, yp, zp);
    }
}

// Tasks of set PH handed out through a shared-memory counter: threads that
// finish their own phase work early (sweep columns, store rows) pick up the
// remaining gather tasks.
template <int ORDER, int PH, bool ROWI = false>
__device__ __forceinline__ void gather_pool(float* sm, const SweepArgs<float>& a, const ItemTab& t, int* cnt) {
    for (;;) {
        const int r = atomicAdd(cnt, 1);
        if (r >= GatherSet<ORDER, PH>::N) break;
        gather_task<ORDER, PH, ROWI>(sm, a, t, r);
    }
}

// Coarse-fine ghost cells of a launch (Sec. 2.2: Min-Mod interpolation from
// the coarser level), formed before its sweeps: one block per ghost slot of
// the levels from lc on, i.e. per group with a region on the coarser
// level, which fills those regions' cells in its slot, a thread per coarse cell
// under them (the padded block spans coarse cells -2..9 per axis: 2, 8, 2
// per region along each axis): the cell, its six neighbours and its three
// limited slopes are read and formed once and give all of its children
// inside the block -- the arithmetic of prolong_cell, child by child.  The
// children of one coarse cell lie in one region (region edges are even in
// fine cells), which decides: a region is filled where its source is the
// coarser level, except x-edges clamped at an outflow face (those repeat
// the centre's edge cell, read from the slot).  The sweep launch that
// follows on the stream copies the slot like same-level ghosts, so no phase
// of a sweep block waits on an interpolation.
constexpr int NT_GHOST = 256;

__global__ void __launch_bounds__(NT_GHOST) k_ghost_f32(const SweepArgs<float> a, int lc) {
    __shared__ ItemTab t;
    __shared__ int s_off[28];          // first task of each region (prefix sums of their coarse cells)
    int l = lc, b = (int)blockIdx.x;
    while (b >= a.lv[l].n_slots) b -= a.lv[l].n_slots, ++l;
    const LevelArgs<float>& L = a.lv[l];
    build_tab(t, a, L.item0 + L.slot_g[b], 0);
    __syncthreads();
    if (threadIdx.x < 32) {
        const int r = threadIdx.x;
        const int rx = r % 3 - 1;
        int n = 0;
        if (r < 27 && r != 13 && t.src[r] < 0 && !(rx != 0 && (t.mask[r] & 1)))
            n = (rx ? 2 : PS) * ((r / 3) % 3 == 1 ? PS : 2) * (r / 9 == 1 ? PS : 2);
        // inclusive warp scan
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int m = __shfl_up_sync(0xffffffffu, n, d);
            if (r >= d) n += m;
        }
        if (r < 27) s_off[r + 1] = n;
        if (r == 0) s_off[0] = 0;
    }
    __syncthreads();
    float* G = L.ghost + (size_t)t.gslot * GHOST_PG;
    const int lp = t.par & 7;
    const int px = PS * (lp & 1), py = PS * ((lp >> 1) & 1), pz = PS * ((lp >> 2) & 1);
    const size_t vs = (size_t)L.n_groups_c * 8 * 512;
    const float w = (float)L.cw;
    for (int i = threadIdx.x; i < s_off[27]; i += NT_GHOST) {
        int r = 0;
        while (s_off[r + 1] <= i) ++r;
        const int rx = r % 3 - 1, ry = (r / 3) % 3 - 1, rz = r / 9 - 1;
        const int nx = rx ? 2 : PS, ny = ry ? 2 : PS;
        const int j = i - s_off[r];
        // region -1: coarse -2, -1; region 0: 0..7; region +1: 8, 9
        const int cx = (rx < 0 ? -2 : (rx > 0 ? PS : 0)) + j % nx;
        const int cy = (ry < 0 ? -2 : (ry > 0 ? PS : 0)) + (j / nx) % ny;
        const int cz = (rz < 0 ? -2 : (rz > 0 ? PS : 0)) + j / (nx * ny);
        // the coarse cell and its six neighbours in the parent's coarse group
        const int X = px + cx, Y = py + cy, Z = pz + cz;
        auto at = [&](int u, int v, int q) -> size_t {
            const int s = resolve(t.csrc, t.cmask, u, v, q);
            return cell_offset(s < 0 ? 0 : s, u, v, q);     // s < 0 cannot pass host validation
        };
        const size_t o[7] = {at(X, Y, Z),     at(X - 1, Y, Z), at(X + 1, Y, Z), at(X, Y - 1, Z),
                             at(X, Y + 1, Z), at(X, Y, Z - 1), at(X, Y, Z + 1)};
        // children inside the padded block: fine 2c + d in [-3, 19)
        const int d0x = cx == -2 ? 1 : 0, d1x = cx == 9 ? 0 : 1;
        const int d0y = cy == -2 ? 1 : 0, d1y = cy == 9 ? 0 : 1;
        const int d0z = cz == -2 ? 1 : 0, d1z = cz == 9 ? 0 : 1;
#pragma unroll 1
        for (int v = 0; v < NV; ++v) {
            const float* p = L.uc + v * vs;
            float c[7];
#pragma unroll
            for (int q = 0; q < 7; ++q) c[q] = p[o[q]];
            if (L.ucn != nullptr) {
                // individual time steps: the coarse state at the start of
                // this level's step, linear in time between before and after
                // the coarse sweep set
                const float* pn = L.ucn + v * vs;
#pragma unroll
                for (int q = 0; q < 7; ++q) c[q] = c[q] + w * (pn[o[q]] - c[q]);
            }
            const float U = c[0];
            const float Sx = minmod_slope(c[1], U, c[2]);
            const float Sy = minmod_slope(c[3], U, c[4]);
            const float Sz = minmod_slope(c[5], U, c[6]);
            float* gv = G + v * GVS;
            for (int dz = d0z; dz <= d1z; ++dz)
                for (int dy = d0y; dy <= d1y; ++dy) {
                    const int fy = 2 * cy + dy, fz = 2 * cz + dz;
                    float* row = gv + ((fz + NG) * PD + (fy + NG)) * GROW;
                    const float sy = dy ? 1.0f : -1.0f, sz = dz ? 1.0f : -1.0f;
                    for (int dx = d0x; dx <= d1x; ++dx) {
                        const int fx = 2 * cx + dx;
                        const float sx = dx ? 1.0f : -1.0f;
                        const float tt = (sx * Sx + sy * Sy) + sz * Sz;
                        row[fx < 0 ? GS + NG + fx : (fx >= GS ? fx + 4 : fx)] = U + 0.25f * tt;
                    }
                }
        }
    }
}

// Double-float (hi, lo) accumulation, error-free in each step (two-sum).
__device__ __forceinline__ void df_add(float& hi, float& lo, float x) {
    const float s = hi + x;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (x - bb);
    hi = s;
}

// Diagnostic accumulators of one thread: the exact speed maximum as the bit
// pattern of a non-negative float (a NaN wins), double-float sums of the
// five variables, the count of bad cells.
struct DiagAcc {
    unsigned smax = 0u;
    float hi[NV] = {0.f, 0.f, 0.f, 0.f, 0.f};
    float lo[NV] = {0.f, 0.f, 0.f, 0.f, 0.f};
    int bad = 0;
    __device__ __forceinline__ void add(const float u[NV], float g, float gm1) {
        float sp, P;
        speed_pressure_f32(u, g, gm1, sp, P);
        smax = max(smax, __float_as_uint(sp));
        bool fin = true;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            df_add(hi[v], lo[v], u[v]);
            fin = fin && isfinite(u[v]);
        }
        bad += (!fin || !(u[0] > 0.0f) || !(P > 0.0f)) ? 1 : 0;
    }
    // warp reduction; lane 0 parks the warp's result in red[warp][12]
    __device__ __forceinline__ void park(float* red) {
        const unsigned full = 0xffffffffu;
#pragma unroll
        for (int w = 16; w > 0; w >>= 1) {
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const float oh = __shfl_xor_sync(full, hi[v], w), ol = __shfl_xor_sync(full, lo[v], w);
                df_add(hi[v], lo[v], oh);
                lo[v] += ol;
            }
        }
        smax = __reduce_max_sync(full, smax);
        bad = __reduce_add_sync(full, bad);
        if ((threadIdx.x & 31) == 0) {
            float* rr = red + (threadIdx.x >> 5) * 12;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                rr[2 * v] = hi[v];
                rr[2 * v + 1] = lo[v];
            }
            rr[10] = __uint_as_float(smax);
            rr[11] = __int_as_float(bad);
        }
    }
};

// The last sweep of a set: 256 interior lines (z-columns for xyz, x-rows
// for zyx), one per thread of warps 0..7.  Right after its line the thread
// writes the 16 finished cells to u_out (x-rows: two aligned 16-byte stores
// per patch row and variable; z-columns: one store per cell and variable,
// coalesced across the warp's consecutive x) and, with diagnostics on,
// accumulates them and parks the warp's result in red.
template <int ORDER, int LIM, bool MASK = false>
__device__ __forceinline__ void sweep_last_store(float* sm, float lam, float g, float gm1, float* flux_g,
                                                 const LevelArgs<float>& L, int grp, bool diag, float* red,
                                                 unsigned fm = 0xFFFu) {
    constexpr int AX = ORDER == 0 ? 2 : 0;
    constexpr int T1 = AX == 0 ? 1 : 0;
    constexpr int T2 = AX == 2 ? 1 : 2;
    constexpr int ST[3] = {1, XP, PD * XP};
    constexpr int S = ST[AX];
    const int c = threadIdx.x;               // < 256
    int i1 = NG + c % GS, i2 = NG + c / GS;  // z-columns: natural order keeps the stores coalesced
    if (ORDER == 1) {
        const unsigned m = __ldg(kLaneZyxS3 + c);
        i1 = m & 255u;
        i2 = m >> 8;
    }
    float* p = sm + i1 * ST[T1] + i2 * ST[T2];
    float* fl = flux_g ? flux_g + AX * (3 * NV * 256) + (i2 - NG) * GS + (i1 - NG) : nullptr;
    if (MASK && !((fm >> (4 * AX + 2 * ((i2 - NG) >> 3) + ((i1 - NG) >> 3))) & 1u)) fl = nullptr;
    column<AX, S, LIM>(p, 0.25f * lam, 0.5f * lam, g, gm1, fl);
    const size_t vstride = (size_t)L.n_groups * 8 * 512;
    DiagAcc acc;
    if (AX == 0) {
        float* o = L.u_out + cell_offset(grp, 0, i1 - NG, i2 - NG);
#pragma unroll 1
        for (int j = 0; j < 4; ++j) {
            float u[4][NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
#pragma unroll
                for (int q = 0; q < 4; ++q) u[q][v] = p[(NG + 4 * j + q) + v * VS];
                *reinterpret_cast<float4*>(o + v * vstride + (j >> 1) * 512 + (j & 1) * 4) =
                    make_float4(u[0][v], u[1][v], u[2][v], u[3][v]);
            }
            if (diag) {
#pragma unroll
                for (int q = 0; q < 4; ++q) acc.add(u[q], g, gm1);
            }
        }
    } else {
        float* o = L.u_out + cell_offset(grp, i1 - NG, i2 - NG, 0);
#pragma unroll 2
        for (int z = 0; z < GS; ++z) {
            float u[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                u[v] = p[(NG + z) * S + v * VS];
                o[v * vstride + (z >> 3) * 2048 + (z & 7) * 64] = u[v];   // patch pz = z / 8, row z % 8
            }
            if (diag) acc.add(u, g, gm1);
        }
    }
    if (diag) acc.park(red);
}

// Combine the parked warp results of one item (threads t0..t0+5) and write
// the item's diagnostics: per-variable FP64 sums, the speed maximum as the bit
// pattern of a double, the bad-cell count.
__device__ __forceinline__ void finish_diag(const DiagSink& d, int item, const float* red, int nwarps,
                                            int t0 = 0) {
    const int t = (int)threadIdx.x - t0;
    if (t < 0) return;
    if (t < NV) {
        double s = 0.0;
        for (int w = 0; w < nwarps; ++w) s += (double)red[w * 12 + 2 * t] + (double)red[w * 12 + 2 * t + 1];
        d.pg_sum[(size_t)item * NV + t] = s;
    } else if (t == NV) {
        unsigned m = 0u;
        int b = 0;
        for (int w = 0; w < nwarps; ++w) {
            m = max(m, __float_as_uint(red[w * 12 + 10]));
            b += __float_as_int(red[w * 12 + 11]);
        }
        d.pg_max[item] = (unsigned long long)__double_as_longlong((double)__uint_as_float(m));
        d.pg_bad[item] = b;
    }
}

// Called by every thread of a CTA once its item loop is over.  Each thread
// makes its own writes visible device-wide, then the CTA counts itself.  The
// last CTA to arrive has every other CTA's results in view and the work
// queue to itself (the others have left their loops): it sets the queue and
// the counter back to zero for the next launch and, with the fused step
// reduction on, combines the per-group results of the whole launch (the
// block's shared memory is free by then).
__device__ __forceinline__ void finish_launch(const SweepArgs<float>& a, float* sm, int* s_last) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) *s_last = atomicAdd(a.done, 1u) == gridDim.x - 1u ? 1 : 0;
    __syncthreads();
    if (*s_last == 0) return;
    __threadfence();
    if (threadIdx.x == 0) {
        *a.queue = 0;
        *a.done = 0u;
        if (a.pair.epoch != nullptr) *a.pair.epoch += 1u;   // every CTA read it before counting out
    }
    if (a.step.out == nullptr) return;
    LevelMeta m;
    m.n_levels = 1;
    m.item0[0] = 0;
    m.n[0] = a.step.n_items;
    m.dh[0] = a.step.dh;
    m.dscale[0] = 1.0;
    double* s_sum = reinterpret_cast<double*>(sm);
    unsigned long long* s_max = reinterpret_cast<unsigned long long*>(s_sum + NV * NT_FIN);
    long long* s_bad = reinterpret_cast<long long*>(s_max + NT_FIN);
    step_reduce(m, a.diag.pg_max, a.diag.pg_sum, a.diag.pg_bad, a.step.cfl, a.step.dt, a.step.update_dt,
                a.step.out, a.step.out_host, a.pair.status, s_sum, s_max, s_bad);
}

// Persistent kernel.  NT = 512 threads (16 warps), one CTA per SM.  Work
// items (level, group) come from an atomic counter, one ahead.  Per item:
//   sweep 1: all warps (for xyz each thread first gathers the centre of its
//            own x-row when yp is in [3,19); sets A and B hold the rest);
//   sweep 2: 352 columns on warps 0..10; warps 11..15 build the next item's
//            region tables, prefetch its interior into L2 and gather its set A;
//   sweep 3: 256 lines on warps 0..7, each thread storing its finished line
//            (and accumulating the diagnostics); warps 8..15 gather set B;
//   zyx only: all warps gather the next item's sets C and D.
// The first item of each CTA is gathered whole.
constexpr int NT_F32 = 512;

template <int ORDER, int LIM, bool ROWI = false>
__device__ __forceinline__ void sweep_first(float* sm, const SweepArgs<float>& a, const ItemTab& t,
                                            float lam, float* flux_g, bool whole = false, unsigned fm = 0xFFFu) {
    if (ORDER == 0) {
        // x-rows (yp, zp); rows with yp in [3,19) get their centre first --
        // with `whole` (the first item of a CTA, nothing gathered before)
        // every thread gathers its entire row: the x-sweep of a row reads
        // that row only, so no barrier has to wait for the others
        const int c = threadIdx.x;
        if (c >= PD * PD) return;
        const int yp = c % PD, zp = c / PD;
        if (whole) gather_row<3, ROWI>(sm, a, t, yp, zp);
        else if (yp >= NG && yp < NG + GS) gather_row<1, ROWI>(sm, a, t, yp, zp);
        float* p = sm + yp * XP + zp * (PD * XP);
        column<0, 1, LIM>(p, 0.25f * lam, 0.5f * lam, a.gamma, a.gm1, flux_slot<0, ROWI>(flux_g, fm, yp, zp));
    } else {
        sweep<ORDER, 0, LIM, ROWI>(sm, lam, a.gamma, a.gm1, flux_g, NT_F32, fm);
    }
}

// ROWI: launches that include a level with a coarser level, whose
// coarse-fine ghost cells k_ghost_f32 formed before the launch; launches
// over level 0 alone have no coarse regions and keep the per-cell fallback,
// whose code is smaller.
template <int ORDER, int LIM, bool ROWI>
__global__ void __launch_bounds__(NT_F32, 1) k_sweep_f32(const SweepArgs<float> args) {
    extern __shared__ float sm[];
    ItemTab* tab = reinterpret_cast<ItemTab*>(sm + NV * VS);     // [2]
    int* s_item = reinterpret_cast<int*>(tab + 2);               // current, next
    int* s_cnt = s_item + 2;                                     // gather-set counters A, B; last-CTA flag
    float* s_red = reinterpret_cast<float*>(s_cnt + 4);          // [8 warps][12]
    const int tid = threadIdx.x;
    const bool diag = args.diag.pg_max != nullptr;

    if (tid == 0) {
        s_item[0] = atomicAdd(args.queue, 1);
        s_item[1] = atomicAdd(args.queue, 1);
        s_cnt[0] = s_cnt[1] = 0;
    }
    __syncthreads();
    do {
        if (s_item[0] >= args.total) break;
        int slot = 0;
        bool first = true;
        build_tab(tab[0], args, s_item[0], 0);
        __syncthreads();
        // the first item whole (xyz: in sweep 1, each thread its own row)
        if (ORDER == 1)
            for (int r = tid; r < PD * PD; r += NT_F32) gather_row<3, ROWI>(sm, args, tab[0], r % PD, r / PD);

        for (;;) {
            // an xyz item after an xyz item needs no barrier here: the last
            // one closed the previous item's store, and each thread's sweep 1
            // reads only its own row (the previous item's diagnostics are
            // combined meanwhile by threads without a row)
            if (ORDER == 1 || first) __syncthreads();
            const int next = s_item[1];
            const bool has_next = next < args.total;
            const ItemTab& cur = tab[slot];
            ItemTab& nxt = tab[slot ^ 1];
            const LevelArgs<float>& L = args.lv[cur.level];
            float* fg = L.flux ? L.flux + (size_t)cur.g * FLUX_PG : nullptr;
            const float lam = cur.lam;
            const int cur_item = cur.item;
            const int cur_g = cur.g;
            // the face-flux columns the fix-ups read: every column in
            // launches over level 0 alone (their kernels stay smaller)
            const unsigned fm = ROWI && fg != nullptr && L.fneed != nullptr ? __ldg(L.fneed + cur_g) : 0xFFFu;

            sweep_first<ORDER, LIM, ROWI>(sm, args, cur, lam, fg, first, fm);
            first = false;
            __syncthreads();
            if (tid < 11 * 32) {
                sweep<ORDER, 1, LIM, ROWI>(sm, lam, args.gamma, args.gm1, fg, 11 * 32, fm);
                if (ROWI && has_next) {
                    // coarse-fine rows make the gather pool long: the sweeping
                    // warps take what is left of it once the tables are built
                    asm volatile("bar.sync 2, 512;" ::: "memory");
                    gather_pool<ORDER, 0, ROWI>(sm, args, nxt, &s_cnt[0]);
                }
            } else if (has_next) {
                build_tab(nxt, args, next, 11 * 32);
                if (tid == 11 * 32) prefetch_item(args, next);
                asm volatile("bar.sync 1, 160;" ::: "memory");      // warps 11..15: tables ready
                if (ROWI) asm volatile("bar.arrive 2, 512;" ::: "memory");
                gather_pool<ORDER, 0, ROWI>(sm, args, nxt, &s_cnt[0]);
            }
            __syncthreads();
            if (tid < 8 * 32) {
                sweep_last_store<ORDER, LIM, ROWI>(sm, lam, args.gamma, args.gm1, fg, L, cur_g, diag, s_red, fm);
                if (tid == 0) {
                    s_item[0] = next;
                    s_item[1] = has_next ? atomicAdd(args.queue, 1) : next;
                }
                if (ROWI && has_next) gather_pool<ORDER, 1, ROWI>(sm, args, nxt, &s_cnt[1]);
            } else if (has_next) {
                gather_pool<ORDER, 1, ROWI>(sm, args, nxt, &s_cnt[1]);
            }
            __syncthreads();
            if (tid == 0) s_cnt[0] = s_cnt[1] = 0;
            if (diag) finish_diag(args.diag, cur_item, s_red, 8, NT_F32 - 6);
            if (!has_next) break;
            slot ^= 1;
            if (ORDER == 1) {
                // sets C (x-edges of the interior rows) and D (their centres, by halves)
                for (int r = tid; r < GS * GS + 2 * GS * GS; r += NT_F32) {
                    if (r < GS * GS) gather_row<2, ROWI>(sm, args, tab[slot], NG + r % GS, NG + r / GS);
                    else gather_task<ORDER, 3, ROWI>(sm, args, tab[slot], r - GS * GS);
                }
            }
        }
    } while (false);
    finish_launch(args, sm, &s_cnt[2]);
}

// ---------------------------------------------------------------- pair launch

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Warp-collective: are the xyz results of group g and of its 26 neighbours
// published in this launch?
__device__ __forceinline__ bool inputs_ready(const SweepArgs<float>& a, int g, unsigned target) {
    const int lane = threadIdx.x & 31;
    int n = -1;
    if (lane < 26) n = a.lv[0].nbr[(size_t)g * 26 + lane];
    else if (lane == 26) n = g;
    const bool ok = n < 0 || ld_acquire_u32(a.pair.ready + n) == target;
    return __all_sync(0xffffffffu, ok);
}

// Warp-collective wait for inputs_ready, bounded (about a second): a wait
// that runs out sets the launch's status word and goes on, and the step
// reports a timeout instead of hanging.
constexpr unsigned PAIR_SPIN_LIMIT = 1u << 21;
__device__ __forceinline__ void wait_inputs(const SweepArgs<float>& a, int g, unsigned target) {
    for (unsigned it = 0;; ++it) {
        if (inputs_ready(a, g, target)) break;
        if (ld_acquire_u32(a.pair.status) != 0u) break;    // an earlier wait gave up: do not wait again
        if (it >= PAIR_SPIN_LIMIT) {
            if ((threadIdx.x & 31) == 0) atomicOr(a.pair.status, 1u);
            break;
        }
        __nanosleep(256);
    }
    __threadfence();
}

// Publish the xyz result of group g.  Its stores were made by other threads
// of the block before a block-wide barrier that precedes this call; the
// fence orders them (cumulatively) before the mark.
__device__ __forceinline__ void publish(const SweepArgs<float>& a, int g, unsigned target) {
    __threadfence();
    if (g != a.pair.hold) st_release_u32(a.pair.ready + g, target);
}

// Pair launch: the xyz set and then the zyx set of one level with the same
// dt (the forward and backward sweep of Sec. 2.2), u -> u_out -> u, in one
// persistent launch.  Items follow the pipelined kernel above, with the
// order taken per item.  A zyx item reads the xyz results of its group and
// of the 26 neighbours, so it starts only once those are published; its
// ghost slabs are gathered alongside the previous item when that item is
// also a zyx item and the inputs are already published, otherwise after it
// (the CTA first publishes its own pending xyz result, so no CTA ever waits
// on itself).  Waits are only for items already claimed by running CTAs,
// and xyz items never wait, so the launch always completes.
template <int LIM>
__global__ void __launch_bounds__(NT_F32, 1) k_sweep_pair(const SweepArgs<float> args) {
    extern __shared__ float sm[];
    ItemTab* tab = reinterpret_cast<ItemTab*>(sm + NV * VS);     // [2]
    int* s_item = reinterpret_cast<int*>(tab + 2);               // current, next (queue indices)
    int* s_cnt = s_item + 2;          // gather-set counters A, B; last-CTA flag; next item deferred
    float* s_red = reinterpret_cast<float*>(s_cnt + 4);          // [8 warps][12]
    int* s_aux = reinterpret_cast<int*>(s_red + 8 * 12);         // pending publication, target mark
    const int tid = threadIdx.x;
    const int total = args.total;
    const bool diag = args.diag.pg_max != nullptr;

    if (tid == 0) {
        s_item[0] = atomicAdd(args.queue, 1);
        s_item[1] = atomicAdd(args.queue, 1);
        s_cnt[0] = s_cnt[1] = 0;
        s_aux[0] = -1;
        s_aux[1] = (int)(ld_acquire_u32(args.pair.epoch) + 1u);
    }
    __syncthreads();
    const unsigned target = (unsigned)s_aux[1];
    do {
        if (s_item[0] >= total) break;
        int slot = 0;
        bool first = true;               // an xyz first item gathers its rows in sweep 1
        build_tab(tab[0], args, s_item[0], 0);
        __syncthreads();
        if (tab[0].level != 0) {
            if (tid < 32) wait_inputs(args, tab[0].g, target);
            __syncthreads();
            for (int r = tid; r < PD * PD; r += NT_F32) gather_row<3>(sm, args, tab[0], r % PD, r / PD);
        }

        for (;;) {
            __syncthreads();
            const int next = s_item[1];
            const bool has_next = next < total;
            const ItemTab& cur = tab[slot];
            ItemTab& nxt = tab[slot ^ 1];
            const int ord = cur.level;                       // 0: xyz, 1: zyx
            const LevelArgs<float>& L = args.lv[ord];
            const float lam = cur.lam;
            const int cur_g = cur.g;

            if (ord == 0) sweep_first<0, LIM>(sm, args, cur, lam, nullptr, first);
            else sweep_first<1, LIM>(sm, args, cur, lam, nullptr);
            first = false;
            __syncthreads();
            if (tid == 11 * 32 && s_aux[0] >= 0) {
                publish(args, s_aux[0], target);       // the previous xyz item
                s_aux[0] = -1;
            }
            if (tid < 11 * 32) {
                if (ord == 0) sweep<0, 1, LIM>(sm, lam, args.gamma, args.gm1, nullptr, 11 * 32);
                else sweep<1, 1, LIM>(sm, lam, args.gamma, args.gm1, nullptr, 11 * 32);
            } else if (has_next) {
                build_tab(nxt, args, next, 11 * 32);
                if (tid == 11 * 32) prefetch_item(args, next);
                asm volatile("bar.sync 1, 160;" ::: "memory");      // warps 11..15: tables ready
                if (tid < 12 * 32) {
                    bool go = nxt.level == ord;
                    if (go && ord == 1) go = inputs_ready(args, nxt.g, target);
                    if (tid == 11 * 32) s_cnt[3] = go ? 0 : 1;
                }
                asm volatile("bar.sync 1, 160;" ::: "memory");
                if (s_cnt[3] == 0) {
                    if (ord == 0) gather_pool<0, 0>(sm, args, nxt, &s_cnt[0]);
                    else gather_pool<1, 0>(sm, args, nxt, &s_cnt[0]);
                }
            }
            __syncthreads();
            if (tid < 8 * 32) {
                if (ord == 0) sweep_last_store<0, LIM>(sm, lam, args.gamma, args.gm1, nullptr, L, cur_g, false, s_red);
                else sweep_last_store<1, LIM>(sm, lam, args.gamma, args.gm1, nullptr, L, cur_g, diag, s_red);
                if (tid == 0) {
                    s_item[0] = next;
                    s_item[1] = has_next ? atomicAdd(args.queue, 1) : next;
                }
            } else if (has_next && s_cnt[3] == 0) {
                if (ord == 0) gather_pool<0, 1>(sm, args, nxt, &s_cnt[1]);
                else gather_pool<1, 1>(sm, args, nxt, &s_cnt[1]);
            }
            __syncthreads();
            if (tid == 0) {
                s_cnt[0] = s_cnt[1] = 0;
                if (ord == 0) s_aux[0] = cur_g;       // published in the next phase 2, or below
            }
            if (ord == 1 && diag) finish_diag(args.diag, cur_g, s_red, 8, NT_F32 - 6);
            if (!has_next) break;
            slot ^= 1;
            if (s_cnt[3] != 0) {
                // a zyx item not gathered alongside: publish our own pending xyz
                // result (the item may need it), wait for its inputs, gather it
                __syncthreads();
                if (tid == 0 && s_aux[0] >= 0) {
                    publish(args, s_aux[0], target);
                    s_aux[0] = -1;
                }
                if (tid < 32) wait_inputs(args, tab[slot].g, target);
                __syncthreads();
                for (int r = tid; r < PD * PD; r += NT_F32) gather_row<3>(sm, args, tab[slot], r % PD, r / PD);
            } else if (ord == 1) {
                for (int r = tid; r < GS * GS + 2 * GS * GS; r += NT_F32) {
                    if (r < GS * GS) gather_row<2>(sm, args, tab[slot], NG + r % GS, NG + r / GS);
                    else gather_task<1, 3>(sm, args, tab[slot], r - GS * GS);
                }
            }
        }
    } while (false);
    __syncthreads();
    if (tid == 0 && s_aux[0] >= 0) publish(args, s_aux[0], target);
    finish_launch(args, sm, &s_cnt[2]);
}

// Non-pipelined variant (an autotuner candidate): per item, all NT threads
// gather the whole padded block, then the three sweeps run with every
// thread, the last one storing its lines; the next item's interior is
// prefetched into L2 one item ahead.  Simpler and without the set
// bookkeeping; it can win when a CTA gets about one item.
template <int ORDER, int LIM, int NT>
__global__ void __launch_bounds__(NT, 1) k_sweep_f32_simple(const SweepArgs<float> args) {
    extern __shared__ float sm[];
    ItemTab* tab = reinterpret_cast<ItemTab*>(sm + NV * VS);
    int* s_item = reinterpret_cast<int*>(tab + 2);
    float* s_red = reinterpret_cast<float*>(s_item + 6);       // s_item[2]: last-CTA flag
    const int tid = threadIdx.x;
    const bool diag = args.diag.pg_max != nullptr;
    if (tid == 0) {
        s_item[0] = atomicAdd(args.queue, 1);
        s_item[1] = atomicAdd(args.queue, 1);
    }
    __syncthreads();
    for (;;) {
        const int item = s_item[0], next = s_item[1];
        if (item >= args.total) break;
        build_tab(tab[0], args, item, 0);
        if (tid == 0 && next < args.total) prefetch_item(args, next);
        __syncthreads();
        const ItemTab& cur = tab[0];
        const LevelArgs<float>& L = args.lv[cur.level];
        float* fg = L.flux ? L.flux + (size_t)cur.g * FLUX_PG : nullptr;
        const float lam = cur.lam;
        const int cur_item = cur.item, cur_g = cur.g;
        for (int r = tid; r < PD * PD; r += NT) gather_row<3>(sm, args, cur, r % PD, r / PD);
        __syncthreads();
        sweep<ORDER, 0, LIM>(sm, lam, args.gamma, args.gm1, fg, NT);
        __syncthreads();
        sweep<ORDER, 1, LIM>(sm, lam, args.gamma, args.gm1, fg, NT);
        __syncthreads();
        if (tid < 8 * 32) sweep_last_store<ORDER, LIM>(sm, lam, args.gamma, args.gm1, fg, L, cur_g, diag, s_red);
        if (tid == 0) {
            s_item[0] = next;
            s_item[1] = next < args.total ? atomicAdd(args.queue, 1) : next;
        }
        __syncthreads();
        if (diag) finish_diag(args.diag, cur_item, s_red, 8);
    }
    finish_launch(args, sm, &s_item[2]);
}

template <typename K>
static cudaError_t set_attr(K k) {
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_F32);
}

// Opt every instantiation into the large dynamic shared memory once per
// process and device (not a stream operation, so it stays out of graph
// capture).
cudaError_t sweep_f32_init() {
    cudaError_t e = cudaSuccess;
    const cudaError_t r[] = {
        set_attr(k_sweep_f32<0, 0, false>), set_attr(k_sweep_f32<0, 1, false>), set_attr(k_sweep_f32<1, 0, false>),
        set_attr(k_sweep_f32<1, 1, false>), set_attr(k_sweep_f32<0, 0, true>), set_attr(k_sweep_f32<0, 1, true>),
        set_attr(k_sweep_f32<1, 0, true>), set_attr(k_sweep_f32<1, 1, true>), set_attr(k_sweep_f32_simple<0, 0, 256>),
        set_attr(k_sweep_f32_simple<0, 1, 256>), set_attr(k_sweep_f32_simple<1, 0, 256>),
        set_attr(k_sweep_f32_simple<1, 1, 256>), set_attr(k_sweep_f32_simple<0, 0, 512>),
        set_attr(k_sweep_f32_simple<0, 1, 512>), set_attr(k_sweep_f32_simple<1, 0, 512>),
        set_attr(k_sweep_f32_simple<1, 1, 512>), set_attr(k_sweep_pair<0>), set_attr(k_sweep_pair<1>)};
    for (cudaError_t x : r)
        if (x != cudaSuccess) e = x;
    return e;
}

template <int ORDER, int LIM>
static cudaError_t launch_pipe(const SweepArgs<float>& a, int grid, cudaStream_t st) {
    int lc = -1;                         // the first level of the launch with a coarser level
    for (int l = a.n_levels - 1; l >= 0; --l)
        if (a.lv[l].uc != nullptr) lc = l;
    if (lc < 0) {
        k_sweep_f32<ORDER, LIM, false><<<grid, NT_F32, SMEM_F32, st>>>(a);
        return cudaGetLastError();
    }
    // every level from lc on has a coarser level and its ghost slot maps
    int n = 0;
    for (int l = lc; l < a.n_levels; ++l) {
        const LevelArgs<float>& L = a.lv[l];
        if (L.n_groups > 0 && (L.uc == nullptr || L.gslot == nullptr || (L.n_slots > 0 && L.slot_g == nullptr)))
            return cudaErrorInvalidValue;
        n += L.n_slots;
    }
    if (n > 0) k_ghost_f32<<<n, NT_GHOST, 0, st>>>(a, lc);
    k_sweep_f32<ORDER, LIM, true><<<grid, NT_F32, SMEM_F32, st>>>(a);
    return cudaGetLastError();
}

template <int ORDER, int LIM, int NT>
static cudaError_t launch_simple(const SweepArgs<float>& a, int grid, cudaStream_t st) {
    k_sweep_f32_simple<ORDER, LIM, NT><<<grid, NT, SMEM_F32, st>>>(a);
    return cudaGetLastError();
}

template <int ORDER, int LIM>
static cudaError_t launch_variant(const SweepArgs<float>& a, int variant, int threads, int grid, cudaStream_t st) {
    if (variant == 0 && threads == NT_F32) return launch_pipe<ORDER, LIM>(a, grid, st);
    if (variant == 1 && threads == 256) return launch_simple<ORDER, LIM, 256>(a, grid, st);
    if (variant == 1 && threads == 512) return launch_simple<ORDER, LIM, 512>(a, grid, st);
    return cudaErrorInvalidValue;
}

size_t sweep_f32_smem() { return SMEM_F32; }

cudaError_t launch_sweep_pair(const SweepArgs<float>& a, int lim, int grid, cudaStream_t st) {
    if (lim == 0) k_sweep_pair<0><<<grid, NT_F32, SMEM_F32, st>>>(a);
    else k_sweep_pair<1><<<grid, NT_F32, SMEM_F32, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sweep_f32(const SweepArgs<float>& a, int order, int lim, int variant, int threads, int grid,
                             cudaStream_t st) {
    if (order == 0) return lim == 0 ? launch_variant<0, 0>(a, variant, threads, grid, st)
                                    : launch_variant<0, 1>(a, variant, threads, grid, st);
    return lim == 0 ? launch_variant<1, 0>(a, variant, threads, grid, st)
                    : launch_variant<1, 1>(a, variant, threads, grid, st);
}

}  // namespace gh
