// sweep_f64.cu -- plain FP64 relaxing-TVD patch-group kernel.
//
// The reference-precision path: one thread block per patch group, as in the
// paper's GPU solver (Sec. 3.1), one launch per chunk of groups.  The padded
// 22^3 x 5 block of a group (425,920 B in FP64, more than a CTA's shared
// memory) is staged in a global scratch buffer owned by the handle; the
// three sweeps update it in place, one thread per 1-D column with a
// register window, and the 16^3 interior is copied to u_out.
//
// Every floating-point operation follows the order of the plain definition
// of the scheme (Eqs. LRFlux, MidpointValue, 2ndTVDFluxCorr..2ndRFlux,
// FullstepValue, vanLeer) with only exact power-of-two rescalings (A = 2F^R,
// B = 2F^L), and this file is compiled with -fmad=false, so a step rounds
// exactly like the plain definition: the FP64 GPU result is meant to be
// bit-identical to a straightforward double-precision evaluation.
#include "common.cuh"
#include "internal.h"

namespace gh {

constexpr int XP64 = PD;
constexpr size_t VS64 = (size_t)PD * PD * PD;
constexpr size_t BLK64 = NV * VS64;   // doubles per staged block

// A = c u + F (= 2 F^R) and B = c u - F (= 2 F^L), Eq. LRFlux with the
// freezing speed c = |v_d| + c_s; pressure from Eqs. ThermalEnergy, EOS.
template <int AXIS>
__device__ __forceinline__ void state64(const double u[NV], double g, double gm1, double A[NV],
                                        double B[NV]) {
    const double rho = u[0];
    const double vx = u[1] / rho, vy = u[2] / rho, vz = u[3] / rho;
    const double eps = u[4] - (0.5 * rho) * ((vx * vx + vy * vy) + vz * vz);
    const double P = gm1 * eps;
    const double cs = sqrt((g * fmax(P, 0.0)) / rho);
    const double vn = AXIS == 0 ? vx : (AXIS == 1 ? vy : vz);
    const double c = fabs(vn) + cs;
    double F[NV];
    F[0] = u[1 + AXIS];
    F[1] = u[1] * vn;
    F[2] = u[2] * vn;
    F[3] = u[3] * vn;
    F[1 + AXIS] = u[1 + AXIS] * vn + P;
    F[4] = (u[4] + P) * vn;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        A[v] = c * u[v] + F[v];
        B[v] = c * u[v] - F[v];
    }
}

// psi(x, y) = 2 phi(x/4, y/4): van Leer 2ab/(a+b) (Eq. vanLeer) or minmod,
// on the unhalved differences of A or B.
template <int LIM>
__device__ __forceinline__ double psi64(double x, double y) {
    if (LIM == 0) {
        if (x * y > 0.0) return (x * y) / (x + y);
        return 0.0;
    } else {
        if (x * y > 0.0) {
            const double m = fmin(fabs(x), fabs(y));
            return 0.5 * (x > 0.0 ? m : -m);
        }
        return 0.0;
    }
}

template <int AXIS, int S, int LIM>
__device__ __forceinline__ void column64(double* __restrict__ p, double lam, double g, double gm1,
                                         double* __restrict__ fl) {
    const double lam_h = 0.5 * lam;    // dt / (2 dx)  (Eq. MidpointValue)
    const double lam_q = 0.25 * lam;   // applied to 2 F
    double u1[NV], u2[NV], u3[NV];
    double Ap[NV], Hp[NV], Aq[NV], Bq[NV], dAp[NV], dBp[NV], Ahp[NV], Gp[NV];
#pragma unroll
    for (int k = 0; k < PD; ++k) {
        double u[NV], A[NV], B[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) u[v] = p[k * S + v * VS64];
        state64<AXIS>(u, g, gm1, A, B);
        if (k >= 1) {
            double H[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) H[v] = Ap[v] - B[v];
            if (k >= 2) {
                double uh[NV], A1[NV], B1[NV];
#pragma unroll
                for (int v = 0; v < NV; ++v) uh[v] = u1[v] - lam_q * (H[v] - Hp[v]);
                state64<AXIS>(uh, g, gm1, A1, B1);
                if (k >= 3) {
                    double dA[NV], dB[NV];
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        dA[v] = A1[v] - Aq[v];
                        dB[v] = B1[v] - Bq[v];
                    }
                    if (k >= 4) {
                        double Ah[NV], Bh[NV];
#pragma unroll
                        for (int v = 0; v < NV; ++v) {
                            Ah[v] = Aq[v] + psi64<LIM>(dAp[v], dA[v]);
                            Bh[v] = Bq[v] - psi64<LIM>(dB[v], dBp[v]);
                        }
                        if (k >= 5) {
                            double Gn[NV];
#pragma unroll
                            for (int v = 0; v < NV; ++v) Gn[v] = Ahp[v] - Bh[v];
                            if ((k == 5 || k == 13 || k == 21) && fl != nullptr) {
#pragma unroll
                                for (int v = 0; v < NV; ++v)
                                    fl[((k - 5) / 8) * (NV * 256) + v * 256] = 0.5 * Gn[v];
                            }
                            if (k >= 6) {
#pragma unroll
                                for (int v = 0; v < NV; ++v)
                                    p[(k - 3) * S + v * VS64] = u3[v] - lam_h * (Gn[v] - Gp[v]);
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

template <int NT, int ORDER, int S_IDX, int LIM>
__device__ __forceinline__ void sweep64(double* blk, double lam, double g, double gm1, double* flux_g) {
    constexpr int AX = ORDER == 0 ? S_IDX : 2 - S_IDX;
    constexpr int T1 = AX == 0 ? 1 : 0;
    constexpr int T2 = AX == 2 ? 1 : 2;
    constexpr bool D1 = ORDER == 0 ? (T1 < AX) : (T1 > AX);
    constexpr bool D2 = ORDER == 0 ? (T2 < AX) : (T2 > AX);
    constexpr int LO1 = D1 ? NG : 0, N1 = D1 ? GS : PD;
    constexpr int LO2 = D2 ? NG : 0, N2 = D2 ? GS : PD;
    constexpr int ST[3] = {1, XP64, PD * XP64};
    constexpr int S = ST[AX];
    for (int c = threadIdx.x; c < N1 * N2; c += NT) {
        const int i1 = LO1 + c % N1, i2 = LO2 + c / N1;
        double* p = blk + i1 * ST[T1] + i2 * ST[T2];
        double* fl = nullptr;
        if (flux_g != nullptr && i1 >= NG && i1 < NG + GS && i2 >= NG && i2 < NG + GS)
            fl = flux_g + AX * (3 * NV * 256) + (i2 - NG) * GS + (i1 - NG);
        column64<AX, S, LIM>(p, lam, g, gm1, fl);
    }
}

// Group g0 + blockIdx.x of level L; scratch block blockIdx.x of `stage`.
template <int ORDER, int LIM, int NT64>
__global__ void __launch_bounds__(NT64) k_pg_f64(const LevelArgs<double> L, int g0, double gamma,
                                                  double gm1, const double* __restrict__ dt,
                                                  double* __restrict__ stage) {
    __shared__ int s_tab[160];
    __shared__ double s_lam;
    if (threadIdx.x == 0) s_lam = (*dt * L.dts) / L.dh;   // lambda = dt / dh (Eq. FullstepValue)
    int* s_src = s_tab;
    int* s_mask = s_tab + 32;
    int* s_csrc = s_tab + 64;
    int* s_cmask = s_tab + 96;
    int* s_par = s_tab + 128;
    const int g = g0 + blockIdx.x;
    double* blk = stage + (size_t)blockIdx.x * BLK64;

    build_tables<double>(L, g, s_src, s_mask, s_csrc, s_cmask, s_par);
    __syncthreads();
    int ppx = 0, ppy = 0, ppz = 0;
    if (*s_par >= 0) {
        const int lp = *s_par & 7;
        ppx = lp & 1; ppy = (lp >> 1) & 1; ppz = (lp >> 2) & 1;
    }
    gather_block<double, XP64, NT64>(blk, VS64, L, g, s_src, s_mask, s_csrc, s_cmask, ppx, ppy, ppz);
    __syncthreads();
    double* fg = L.flux ? L.flux + (size_t)g * FLUX_PG : nullptr;
    sweep64<NT64, ORDER, 0, LIM>(blk, s_lam, gamma, gm1, fg);
    __syncthreads();
    sweep64<NT64, ORDER, 1, LIM>(blk, s_lam, gamma, gm1, fg);
    __syncthreads();
    sweep64<NT64, ORDER, 2, LIM>(blk, s_lam, gamma, gm1, fg);
    __syncthreads();
    const size_t vstride = (size_t)L.n_groups * 8 * 512;
    double* out = L.u_out + ((size_t)g << 12);
    for (int i = threadIdx.x; i < CELLS_PG; i += NT64) {
        const int patch = i >> 9, w = i & 511;
        const int x = ((patch & 1) << 3) | (w & 7);
        const int y = (((patch >> 1) & 1) << 3) | ((w >> 3) & 7);
        const int z = ((patch >> 2) << 3) | (w >> 6);
        const double* s = blk + ((size_t)(z + NG) * PD + (y + NG)) * XP64 + (x + NG);
#pragma unroll
        for (int v = 0; v < NV; ++v) out[v * vstride + i] = s[v * VS64];
    }
}

size_t stage_f64_bytes_per_group() { return BLK64 * sizeof(double); }

template <int NT>
static cudaError_t launch_nt(const LevelArgs<double>& L, int g0, int count, int order, int lim, double gamma,
                             double gm1, const double* dt, double* stage, cudaStream_t st) {
    if (order == 0) {
        if (lim == 0) k_pg_f64<0, 0, NT><<<count, NT, 0, st>>>(L, g0, gamma, gm1, dt, stage);
        else k_pg_f64<0, 1, NT><<<count, NT, 0, st>>>(L, g0, gamma, gm1, dt, stage);
    } else {
        if (lim == 0) k_pg_f64<1, 0, NT><<<count, NT, 0, st>>>(L, g0, gamma, gm1, dt, stage);
        else k_pg_f64<1, 1, NT><<<count, NT, 0, st>>>(L, g0, gamma, gm1, dt, stage);
    }
    return cudaGetLastError();
}

cudaError_t launch_pg_f64(const LevelArgs<double>& L, int g0, int count, int order, int lim,
                          double gamma, double gm1, const double* dt, double* stage, int threads,
                          cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    if (threads == 128) return launch_nt<128>(L, g0, count, order, lim, gamma, gm1, dt, stage, st);
    if (threads == 256) return launch_nt<256>(L, g0, count, order, lim, gamma, gm1, dt, stage, st);
    return cudaErrorInvalidValue;
}

}  // namespace gh
