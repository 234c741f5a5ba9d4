// poisson.cu -- red-black SOR Poisson solver of the refined levels (Sec.
// 2.3, Eqs. DiscretePoisson, Residual, SOR; Sec. 3.2): one thread block per
// patch group, the whole 18^3 potential block (16^3 interior + the
// Dirichlet ghost layer) in shared memory for all iterations -- on GB300 it
// fits with room to spare, where the paper had to split it between shared
// memory and registers.  Each thread owns one interior x-row: its 16 cells,
// their two x-ghosts and 4 pi G dh^2 rho of the row stay in registers, so
// an update reads only its four y and z neighbours from shared memory and
// writes its new value back for the neighbouring rows.  Compiled with
// -fmad=false: the FP64 path evaluates Eqs. Residual and SOR in the
// oracle's order.
#include <cstdint>
#include <string>

#include "gamer_hydro.h"
#include "internal.h"

namespace gh {

constexpr int PP = GS + 2;            // 18 cells per row of the block
constexpr int PL = PP * PP + 1;       // plane pitch: odd, so that the four planes of a warp use disjoint banks
constexpr int NT_SOR = 256;           // one thread per interior x-row
constexpr int HR = GS / 2;            // cells of one colour in a row

// One half-step of a thread's row: the cells with x parity I0 (warp-uniform,
// the warps being grouped by the parity of j + k), in increasing x.  re/ro:
// the row's even-x / odd-x cells; gl, gr: its x-ghosts; cre/cro: 4 pi G dh^2
// rho of the even-x / odd-x cells.  The six neighbours are summed in the
// order x+, y+, z+, x-, y-, z- (Eq. Residual), then phi += (omega/6) R (Eq.
// SOR).
template <int I0, bool CHECK, typename T>
__device__ __forceinline__ void sor_half(T* __restrict__ s, int row, T (&re)[HR], T (&ro)[HR], T gl, T gr,
                                         const T (&cre)[HR], const T (&cro)[HR], T w6, T& norm) {
#pragma unroll
    for (int q = 0; q < HR; ++q) {
        const int c = row + I0 + 2 * q;
        const T cur = I0 ? ro[q] : re[q];
        const T xp = I0 ? (q + 1 < HR ? re[q + 1] : gr) : ro[q];
        const T xm = I0 ? re[q] : (q > 0 ? ro[q - 1] : gl);
        const T nb = ((((xp + s[c + PP]) + s[c + PL]) + xm) + s[c - PP]) + s[c - PL];
        const T R = (nb - T(6) * cur) - (I0 ? cro[q] : cre[q]);
        const T nv = cur + w6 * R;
        if (I0) ro[q] = nv;
        else re[q] = nv;
        s[c] = nv;
        if (CHECK) norm += fabs(R);
    }
}

template <typename T, bool CHECK>
__global__ void __launch_bounds__(NT_SOR) k_sor(const T* __restrict__ rho, T* __restrict__ phi, T coef,
                                                T w6, int max_iter, double tol, int* iters) {
    extern __shared__ unsigned char sraw[];
    T* s = reinterpret_cast<T*>(sraw);                         // [18 planes of PL][18][18]
    __shared__ double s_red[NT_SOR / 32];
    __shared__ int s_stop;
    const int g = blockIdx.x, t = threadIdx.x;
    T* gphi = phi + (size_t)g * PP * PP * PP;
    for (int i = t; i < PP * PP * PP; i += NT_SOR) s[(i / (PP * PP)) * PL + i % (PP * PP)] = gphi[i];
    // rows with j + k even on warps 0..3, odd on warps 4..7
    const int par = t >> 7, r = t & 127;
    const int k = r >> 3, j = 2 * (r & 7) + ((k + par) & 1);
    const int row = (k + 1) * PL + (j + 1) * PP + 1;           // cell (0, j, k) of the row
    T cre[HR], cro[HR];
    const T* rrow = rho + ((size_t)g * GS + k) * GS * GS + j * GS;
#pragma unroll
    for (int q = 0; q < HR; ++q) {
        cre[q] = coef * rrow[2 * q];
        cro[q] = coef * rrow[2 * q + 1];
    }
    double src_all = 0.0;
    if (CHECK) {
        // one-norm of the source, block-wide
        T src = T(0);
#pragma unroll
        for (int q = 0; q < HR; ++q) src += fabs(cre[q]) + fabs(cro[q]);
        for (int o = 16; o > 0; o >>= 1) src += __shfl_xor_sync(0xffffffffu, src, o);
        if ((t & 31) == 0) s_red[t >> 5] = (double)src;
    }
    __syncthreads();
    if (CHECK) {
        for (int w = 0; w < NT_SOR / 32; ++w) src_all += s_red[w];
        __syncthreads();
    }
    T re[HR], ro[HR];
#pragma unroll
    for (int q = 0; q < HR; ++q) {
        re[q] = s[row + 2 * q];
        ro[q] = s[row + 2 * q + 1];
    }
    const T gl = s[row - 1], gr = s[row + GS];
    int it = 0;
    while (it < max_iter) {
        T norm = T(0);                                         // residual one-norm, in the data's precision
#pragma unroll
        for (int color = 0; color < 2; ++color) {
            // x parity of this colour's cells: (i + j + k) & 1 == color
            if (((color + par) & 1) == 0) sor_half<0, CHECK>(s, row, re, ro, gl, gr, cre, cro, w6, norm);
            else sor_half<1, CHECK>(s, row, re, ro, gl, gr, cre, cro, w6, norm);
            __syncthreads();
        }
        ++it;
        if (CHECK) {
            for (int o = 16; o > 0; o >>= 1) norm += __shfl_xor_sync(0xffffffffu, norm, o);
            if ((t & 31) == 0) s_red[t >> 5] = (double)norm;
            __syncthreads();
            if (t == 0) {
                double n = 0.0;
                for (int w = 0; w < NT_SOR / 32; ++w) n += s_red[w];
                s_stop = n <= tol * src_all;
            }
            __syncthreads();
            if (s_stop) break;
        }
    }
    for (int i = t; i < PP * PP * PP; i += NT_SOR) gphi[i] = s[(i / (PP * PP)) * PL + i % (PP * PP)];
    if (iters != nullptr && t == 0) iters[g] = it;
}

template <typename T>
static cudaError_t launch_sor(int n, const T* rho, T* phi, double coef, double omega, int max_iter, double tol,
                              int* iters, cudaStream_t st) {
    const size_t smem = sizeof(T) * PP * PL;
    const bool check = tol > 0.0;                              // tol = 0: no norms at all
    cudaError_t e = check ? cudaFuncSetAttribute(k_sor<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                          : cudaFuncSetAttribute(k_sor<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (check) k_sor<T, true><<<n, NT_SOR, smem, st>>>(rho, phi, (T)coef, (T)(omega / 6.0), max_iter, tol, iters);
    else k_sor<T, false><<<n, NT_SOR, smem, st>>>(rho, phi, (T)coef, (T)(omega / 6.0), max_iter, tol, iters);
    return cudaGetLastError();
}

// Inputs of a refined level's SOR problem (Sec. 2.3; reading R26), one
// block per patch group: every cell of the 18^3 potential block -- the
// one-cell ghost layer (Dirichlet data) and the interior (initial guess) --
// by the Min-Mod interpolation of the coarser level's potential (the same
// arithmetic as the ghost interpolation of the hydro gathers, on one
// variable), and the group's density as a 16^3 block, both x fastest.
constexpr int NT_PREP = 384;          // one thread per (x, y) of an 18 x 18 plane of the block

// The coarse cells the group's interpolation reads -- its parent patch and
// two coarse cells around it, 12^3 -- are staged in shared memory first (all
// loads of a thread in flight together).  The limited slopes of the 10^3
// coarse cells whose children fill the block are then formed once per coarse
// cell, and every fine cell reads its coarse value and three slopes.
constexpr int CW = PS + 4;            // 12 coarse cells per axis
constexpr int CF = PS + 2;            // 10 coarse cells per axis with children in the block

template <typename T>
__global__ void __launch_bounds__(NT_PREP) k_poisson_prepare(const PrepArgs<T> a) {
    __shared__ int s_csrc[27], s_cmask[27];
    __shared__ T s_c[CW * CW * CW];
    __shared__ T s_sl[3][CF * CF * CF];
    const int g = blockIdx.x, t = threadIdx.x;
    const int P = a.parent[g];
    if (t < 27) region_entry(a.nbrc, P >> 3, t, s_csrc, s_cmask);
    __syncthreads();
    const int lp = P & 7;
    const int px = lp & 1, py = (lp >> 1) & 1, pz = (lp >> 2) & 1;
    const int ox = PS * px - 2, oy = PS * py - 2, oz = PS * pz - 2;   // coarse origin of the staged cube
    constexpr int NS = CW * CW * CW;
    constexpr int PER = (NS + NT_PREP - 1) / NT_PREP;
    T v[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = k * NT_PREP + t;
        if (i < NS) {
            int xa = ox + i % CW, ya = oy + (i / CW) % CW, za = oz + i / (CW * CW);
            // proper nesting puts the whole cube in existing coarse patches;
            // a region that did not resolve would only be left unread
            const int s = resolve(s_csrc, s_cmask, xa, ya, za);
            v[k] = s < 0 ? T(0) : a.phi_c[cell_offset(s, xa, ya, za)];
        }
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = k * NT_PREP + t;
        if (i < NS) s_c[i] = v[k];
    }
    __syncthreads();
    // slopes of the coarse cells -1 .. 8 of the parent patch (cube index + 2)
    for (int i = t; i < CF * CF * CF; i += NT_PREP) {
        const int cx = i % CF, cy = (i / CF) % CF, cz = i / (CF * CF);
        const int c0 = ((cz + 1) * CW + (cy + 1)) * CW + (cx + 1);
        const T U = s_c[c0];
        s_sl[0][i] = minmod_slope(s_c[c0 - 1], U, s_c[c0 + 1]);
        s_sl[1][i] = minmod_slope(s_c[c0 - CW], U, s_c[c0 + CW]);
        s_sl[2][i] = minmod_slope(s_c[c0 - CW * CW], U, s_c[c0 + CW * CW]);
    }
    __syncthreads();
    // thread t < 18^2 fills column (x, y) = (t % 18 - 1, t / 18 - 1) of the
    // block plane by plane (group-local coordinates -1 .. 16); the coarse
    // cell of a fine cell is (x >> 1, ...) of the parent patch
    T* out = a.phi_blk + (size_t)g * PP * PP * PP;
    if (t < PP * PP) {
        const int x = t % PP - 1, y = t / PP - 1;
        const int cx = (x >> 1) + 1, cy = (y >> 1) + 1;
        const T sx = (x & 1) ? T(1) : T(-1), sy = (y & 1) ? T(1) : T(-1);
#pragma unroll 2
        for (int zz = 0; zz < PP; ++zz) {
            const int z = zz - 1, cz = (z >> 1) + 1;
            const int cf = (cz * CF + cy) * CF + cx;
            const T U = s_c[((cz + 1) * CW + (cy + 1)) * CW + (cx + 1)];
            const T Sx = s_sl[0][cf], Sy = s_sl[1][cf], Sz = s_sl[2][cf];
            const T sz = (z & 1) ? T(1) : T(-1);
            const T tt = (sx * Sx + sy * Sy) + sz * Sz;
            out[zz * PP * PP + t] = U + T(0.25) * tt;
        }
    }
    // density block, x fastest: the group's cells read in their storage order
    // four at a time (one aligned quad of a patch row) and written as a quad
    T* rb = a.rho_blk + (size_t)g * CELLS_PG;
    const T* ug = a.u + ((size_t)g << 12);
    for (int j = 4 * t; j < CELLS_PG; j += 4 * NT_PREP) {
        const int patch = j >> 9, w = j & 511;
        const int x = ((patch & 1) << 3) | (w & 7);
        const int y = (((patch >> 1) & 1) << 3) | ((w >> 3) & 7);
        const int z = ((patch >> 2) << 3) | (w >> 6);
        T* d = rb + (z * GS + y) * GS + x;
#pragma unroll
        for (int q = 0; q < 4; ++q) d[q] = ug[j + q];
    }
}

template <typename T>
cudaError_t launch_poisson_prepare(const PrepArgs<T>& a, cudaStream_t st) {
    if (a.n <= 0) return cudaSuccess;
    k_poisson_prepare<T><<<a.n, NT_PREP, 0, st>>>(a);
    return cudaGetLastError();
}
template cudaError_t launch_poisson_prepare<float>(const PrepArgs<float>&, cudaStream_t);
template cudaError_t launch_poisson_prepare<double>(const PrepArgs<double>&, cudaStream_t);

}  // namespace gh

using namespace gh;

extern "C" int gamer_poisson_sor(int precision, int n_groups, const void* rho, void* phi, double coef, double omega,
                                 int max_iter, double tol, int32_t* iters, void* cuda_stream) {
    auto fail = [](int code, const char* msg) {
        set_thread_error(msg);
        return code;
    };
    if (precision != GAMER_FP32 && precision != GAMER_FP64) return fail(GAMER_ERR_ARG, "unknown precision");
    if (n_groups < 0 || max_iter < 0) return fail(GAMER_ERR_ARG, "negative n_groups or max_iter");
    if (!(omega > 0.0 && omega < 2.0)) return fail(GAMER_ERR_ARG, "omega must be in (0, 2)");
    if (!(tol >= 0.0)) return fail(GAMER_ERR_ARG, "tol must be non-negative");
    if (n_groups == 0) return GAMER_OK;
    if (!rho || !phi) return fail(GAMER_ERR_ARG, "rho and phi are required");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = precision == GAMER_FP32
                        ? launch_sor<float>(n_groups, static_cast<const float*>(rho), static_cast<float*>(phi), coef,
                                            omega, max_iter, tol, iters, st)
                        : launch_sor<double>(n_groups, static_cast<const double*>(rho), static_cast<double*>(phi),
                                             coef, omega, max_iter, tol, iters, st);
    if (e != cudaSuccess) return fail(GAMER_ERR_CUDA, (std::string("SOR launch: ") + cudaGetErrorString(e)).c_str());
    return GAMER_OK;
}
