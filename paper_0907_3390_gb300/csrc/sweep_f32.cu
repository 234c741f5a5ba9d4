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

namespace gh {

constexpr int XP = 23;                    // x pitch: odd, so x-sweep columns hit distinct banks
constexpr int VS = PD * PD * XP;          // floats per variable in shared memory
constexpr size_t SMEM_F32 = (size_t)NV * VS * sizeof(float) + 256 * sizeof(int);

// A = c u + F and B = c u - F of one cell, sweep along AXIS.
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

template <int LIM>
__device__ __forceinline__ float psi(float x, float y) {
    const float p = x * y;
    if (LIM == 0) {
        const float q = __fdividef(p, x + y);
        return p > 0.0f ? q : 0.0f;
    } else {
        const float m = 0.5f * fminf(fabsf(x), fabsf(y));
        return p > 0.0f ? copysignf(m, x) : 0.0f;
    }
}

// One 1-D column of 22 cells starting at p (stride S between cells, VS
// between variables) along AXIS; cells 3..18 are overwritten with the
// full-step values.  fl: face-flux slot of this row ([3 planes][5][256]
// with plane stride 5*256), or nullptr.
template <int AXIS, int S, int LIM>
__device__ __forceinline__ void column(float* __restrict__ p, float lam4, float lam2, float g,
                                       float gm1, float* __restrict__ fl) {
    float u1[NV], u2[NV], u3[NV];          // u_{k-1}, u_{k-2}, u_{k-3}
    float Ap[NV];                          // A_{k-1}
    float Hp[NV];                          // half-step flux at k-3/2 (x2)
    float Aq[NV], Bq[NV];                  // A', B' of the midpoint state at k-2
    float dAp[NV], dBp[NV];                // dA', dB' at k-5/2
    float Ahp[NV];                         // A'_{n+1/2} at k-5/2
    float Gp[NV];                          // net flux (x2) at k-7/2
#pragma unroll
    for (int k = 0; k < PD; ++k) {
        float u[NV], A[NV], B[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) u[v] = p[k * S + v * VS];
        state<AXIS>(u, g, gm1, A, B);
        if (k >= 1) {
            float H[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) H[v] = Ap[v] - B[v];
            if (k >= 2) {
                float uh[NV], A1[NV], B1[NV];
#pragma unroll
                for (int v = 0; v < NV; ++v) uh[v] = fmaf(-lam4, H[v] - Hp[v], u1[v]);
                state<AXIS>(uh, g, gm1, A1, B1);
                if (k >= 3) {
                    float dA[NV], dB[NV];
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        dA[v] = A1[v] - Aq[v];
                        dB[v] = B1[v] - Bq[v];
                    }
                    if (k >= 4) {
                        float Ah[NV], Bh[NV];
#pragma unroll
                        for (int v = 0; v < NV; ++v) {
                            Ah[v] = Aq[v] + psi<LIM>(dAp[v], dA[v]);
                            Bh[v] = Bq[v] - psi<LIM>(dB[v], dBp[v]);
                        }
                        if (k >= 5) {
                            float Gn[NV];
#pragma unroll
                            for (int v = 0; v < NV; ++v) Gn[v] = Ahp[v] - Bh[v];
                            if ((k == 5 || k == 13 || k == 21) && fl != nullptr) {
#pragma unroll
                                for (int v = 0; v < NV; ++v)
                                    fl[((k - 5) / 8) * (NV * 256) + v * 256] = 0.5f * Gn[v];
                            }
                            if (k >= 6) {
#pragma unroll
                                for (int v = 0; v < NV; ++v)
                                    p[(k - 3) * S + v * VS] = fmaf(-lam2, Gn[v] - Gp[v], u3[v]);
                            }
#pragma unroll
                            for (int v = 0; v < NV; ++v) Gp[v] = Gn[v];
                        }
#pragma unroll
                        for (int v = 0; v < NV; ++v) Ahp[v] = Ah[v];
                    }
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        dAp[v] = dA[v];
                        dBp[v] = dB[v];
                    }
                }
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    Aq[v] = A1[v];
                    Bq[v] = B1[v];
                }
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) Hp[v] = H[v];
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            Ap[v] = A[v];
            u3[v] = u2[v];
            u2[v] = u1[v];
            u1[v] = u[v];
        }
    }
}

// Sweep s (0,1,2) of order ORDER over the shared block; columns whose
// transverse axes were swept earlier in this set only cover [3,19).
template <int NT, int ORDER, int S_IDX, int LIM>
__device__ __forceinline__ void sweep(float* sm, float lam, float g, float gm1, float* flux_g) {
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
    for (int c = threadIdx.x; c < N1 * N2; c += NT) {
        const int i1 = LO1 + c % N1, i2 = LO2 + c / N1;
        float* p = sm + i1 * ST[T1] + i2 * ST[T2];
        float* fl = nullptr;
        if (flux_g != nullptr && i1 >= NG && i1 < NG + GS && i2 >= NG && i2 < NG + GS)
            fl = flux_g + AX * (3 * NV * 256) + (i2 - NG) * GS + (i1 - NG);
        column<AX, S, LIM>(p, lam4, lam2, g, gm1, fl);
    }
}

template <int NT, int ORDER, int LIM>
__global__ void __launch_bounds__(NT, 1) k_sweep_f32(const SweepArgs<float> args) {
    extern __shared__ float sm[];
    int* s_int = reinterpret_cast<int*>(sm + NV * VS);
    int* s_src = s_int;          // [27]
    int* s_mask = s_int + 32;    // [27]
    int* s_csrc = s_int + 64;    // [27]
    int* s_cmask = s_int + 96;   // [27]
    int* s_par = s_int + 128;    // parent patch
    int* s_item = s_int + 129;   // current work item

    for (;;) {
        if (threadIdx.x == 0) *s_item = atomicAdd(args.queue, 1);
        __syncthreads();
        const int item = *s_item;
        if (item >= args.total) break;
        int l = 0;
        while (l + 1 < args.n_levels && item >= args.lv[l + 1].item0) ++l;
        const LevelArgs<float>& L = args.lv[l];
        const int g = item - L.item0;

        build_tables<float>(L, g, s_src, s_mask, s_csrc, s_cmask, s_par);
        __syncthreads();
        int ppx = 0, ppy = 0, ppz = 0;
        if (*s_par >= 0) {
            const int lp = *s_par & 7;
            ppx = lp & 1; ppy = (lp >> 1) & 1; ppz = (lp >> 2) & 1;
        }
        gather_block<float, XP, NT>(sm, VS, L, g, s_src, s_mask, s_csrc, s_cmask, ppx, ppy, ppz);
        __syncthreads();

        float* fg = L.flux ? L.flux + (size_t)g * FLUX_PG : nullptr;
        sweep<NT, ORDER, 0, LIM>(sm, L.lam, args.gamma, args.gm1, fg);
        __syncthreads();
        sweep<NT, ORDER, 1, LIM>(sm, L.lam, args.gamma, args.gm1, fg);
        __syncthreads();
        sweep<NT, ORDER, 2, LIM>(sm, L.lam, args.gamma, args.gm1, fg);
        __syncthreads();

        // interior -> u_out, coalesced along patch rows
        const size_t vstride = (size_t)L.n_groups * 8 * 512;
        float* out = L.u_out + ((size_t)g << 12);
        for (int i = threadIdx.x; i < CELLS_PG; i += NT) {
            // i enumerates the group's 8 patches in storage order
            const int patch = i >> 9, w = i & 511;
            const int x = ((patch & 1) << 3) | (w & 7);
            const int y = (((patch >> 1) & 1) << 3) | ((w >> 3) & 7);
            const int z = ((patch >> 2) << 3) | (w >> 6);
            const float* s = sm + ((z + NG) * PD + (y + NG)) * XP + (x + NG);
#pragma unroll
            for (int v = 0; v < NV; ++v) out[v * vstride + i] = s[v * VS];
        }
        __syncthreads();
    }
}

template <int NT, int ORDER, int LIM>
static cudaError_t launch_one(const SweepArgs<float>& a, int grid, cudaStream_t st) {
    auto k = k_sweep_f32<NT, ORDER, LIM>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_F32);
    if (e != cudaSuccess) return e;
    k<<<grid, NT, SMEM_F32, st>>>(a);
    return cudaGetLastError();
}

template <int NT>
static cudaError_t launch_nt(const SweepArgs<float>& a, int order, int lim, int grid, cudaStream_t st) {
    if (order == 0) return lim == 0 ? launch_one<NT, 0, 0>(a, grid, st) : launch_one<NT, 0, 1>(a, grid, st);
    return lim == 0 ? launch_one<NT, 1, 0>(a, grid, st) : launch_one<NT, 1, 1>(a, grid, st);
}

size_t sweep_f32_smem() { return SMEM_F32; }

cudaError_t launch_sweep_f32(const SweepArgs<float>& a, int order, int lim, int threads, int grid,
                             cudaStream_t st) {
    switch (threads) {
        case 256: return launch_nt<256>(a, order, lim, grid, st);
        case 384: return launch_nt<384>(a, order, lim, grid, st);
        case 512: return launch_nt<512>(a, order, lim, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gh
