// poisson.cu -- red-black SOR Poisson solver of the refined levels (Sec.
// 2.3, Eqs. DiscretePoisson, Residual, SOR; Sec. 3.2): one thread block per
// patch group, the whole 18^3 potential block (16^3 interior + the
// Dirichlet ghost layer) in shared memory for all iterations -- on GB300 it
// fits with room to spare, where the paper had to split it between shared
// memory and registers -- and each thread owning one interior x-row, whose
// 8 even and 8 odd cells it updates in the two half-steps, with 4 pi G dh^2
// rho of its 16 cells in registers.  Compiled with -fmad=false: the FP64
// path evaluates Eqs. Residual and SOR in the oracle's order.
#include <cstdint>
#include <string>

#include "gamer_hydro.h"
#include "internal.h"

namespace gh {

constexpr int PP = GS + 2;            // 18
constexpr int NT_SOR = 256;           // one thread per interior x-row

template <typename T>
__global__ void __launch_bounds__(NT_SOR) k_sor(const T* __restrict__ rho, T* __restrict__ phi, T coef,
                                                T w6, int max_iter, double tol, int* iters) {
    extern __shared__ unsigned char sraw[];
    T* s = reinterpret_cast<T*>(sraw);                         // [18][18][18]
    __shared__ double s_red[NT_SOR / 32];
    __shared__ int s_stop;
    const int g = blockIdx.x, t = threadIdx.x;
    T* gphi = phi + (size_t)g * PP * PP * PP;
    for (int i = t; i < PP * PP * PP; i += NT_SOR) s[i] = gphi[i];
    const int j = t % GS, k = t / GS;                          // this thread's row
    T cre[GS / 2], cro[GS / 2];                                // even-x and odd-x cells of the row
    double src = 0.0;
    const T* rrow = rho + ((size_t)g * GS + k) * GS * GS + j * GS;
#pragma unroll
    for (int q = 0; q < GS / 2; ++q) {
        cre[q] = coef * rrow[2 * q];
        cro[q] = coef * rrow[2 * q + 1];
        src += fabs((double)cre[q]);
        src += fabs((double)cro[q]);
    }
    // one-norm of the source, block-wide (order-independent within rounding)
    for (int o = 16; o > 0; o >>= 1) src += __shfl_xor_sync(0xffffffffu, src, o);
    if ((t & 31) == 0) s_red[t >> 5] = src;
    __syncthreads();
    double src_all = 0.0;
    for (int w = 0; w < NT_SOR / 32; ++w) src_all += s_red[w];
    __syncthreads();
    const int row = ((k + 1) * PP + (j + 1)) * PP + 1;         // cell (0, j, k) of the row
    const bool check = tol > 0.0;                              // tol = 0: no norms at all
    int it = 0;
    while (it < max_iter) {
        T norm = T(0);                                         // residual one-norm, in the data's precision
#pragma unroll
        for (int color = 0; color < 2; ++color) {
            const int i0 = (color + j + k) & 1;                // first x of this colour in the row
#pragma unroll
            for (int q = 0; q < GS / 2; ++q) {
                const int i = i0 + 2 * q;
                const int c = row + i;
                const T nb = ((((s[c + 1] + s[c + PP]) + s[c + PP * PP]) + s[c - 1]) + s[c - PP]) + s[c - PP * PP];
                const T R = (nb - T(6) * s[c]) - (i0 ? cro[q] : cre[q]);
                s[c] = s[c] + w6 * R;
                norm += fabs(R);
            }
            __syncthreads();
        }
        ++it;
        if (!check) continue;
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
    for (int i = t; i < PP * PP * PP; i += NT_SOR) gphi[i] = s[i];
    if (iters != nullptr && t == 0) iters[g] = it;
}

template <typename T>
static cudaError_t launch_sor(int n, const T* rho, T* phi, double coef, double omega, int max_iter, double tol,
                              int* iters, cudaStream_t st) {
    const size_t smem = sizeof(T) * PP * PP * PP;
    cudaError_t e = cudaFuncSetAttribute(k_sor<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_sor<T><<<n, NT_SOR, smem, st>>>(rho, phi, (T)coef, (T)(omega / 6.0), max_iter, tol, iters);
    return cudaGetLastError();
}

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
