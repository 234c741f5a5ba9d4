// gravity.cu -- the gravity operator G of the split scheme (Sec. 2.3): the
// Euler equations' gravity source terms (Eqs. MomConserve and
// EnergyConserve with their flux terms dropped) applied to one level for a
// time step, with the cell-centred acceleration from the 3-point central
// difference of the potential.  The hydro sweeps and G alternate in the
// order xyzGGzyx, the two G of one double step taken as one G of twice the
// step.  Compiled with -fmad=false: the FP64 path evaluates the update in
// the oracle's order.
//
// One thread per cell, threads in the level's memory order, so that the
// five state loads and four stores of a warp are whole 128-byte lines; the
// six potential values of a cell come from the group's 18^3 block, whose
// rows neighbouring warps share through L1.  HBM-bound: 20 B read + 16 B
// written + about 5.7 B of potential per cell in FP32.
#include <cmath>
#include <cstdint>
#include <string>

#include "gamer_hydro.h"
#include "internal.h"

namespace gh {

constexpr int NT_GRAV = 256;
constexpr int PB = GS + 2;            // 18: potential block with one ghost layer

// Per cell, along each axis k: d_k = (phi(-1) - phi(+1)) lam (= g_k dt,
// lam = dt / (2 dh)); m_k += rho d_k; e += 0.5 (((m_x + m'_x) d_x +
// (m_y + m'_y) d_y) + (m_z + m'_z) d_z), m' the new momentum -- the exact
// solution of the split equations over the step, with rho and g constant,
// so the thermal energy does not change.
template <typename T>
__global__ void __launch_bounds__(NT_GRAV) k_gravity(T* __restrict__ u, const T* __restrict__ phi,
                                                     int n_groups, T lam) {
    const size_t vs = (size_t)n_groups * CELLS_PG;
    for (size_t i = (size_t)blockIdx.x * NT_GRAV + threadIdx.x; i < vs; i += (size_t)gridDim.x * NT_GRAV) {
        const int g = (int)(i >> 12), j = (int)(i & (CELLS_PG - 1));
        const int p = j >> 9;
        const int x = ((p & 1) << 3) | (j & 7), y = (((p >> 1) & 1) << 3) | ((j >> 3) & 7),
                  z = ((p >> 2) << 3) | ((j >> 6) & 7);
        const T* ph = phi + (size_t)g * (PB * PB * PB) + ((z + 1) * PB + (y + 1)) * PB + (x + 1);
        const T rho = u[i];
        T d[3], m0[3], m1[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int st = k == 0 ? 1 : k == 1 ? PB : PB * PB;
            d[k] = (__ldg(ph - st) - __ldg(ph + st)) * lam;
            m0[k] = u[(1 + k) * vs + i];
        }
        const T e0 = u[4 * vs + i];
#pragma unroll
        for (int k = 0; k < 3; ++k) m1[k] = m0[k] + rho * d[k];
        const T de = ((m0[0] + m1[0]) * d[0] + (m0[1] + m1[1]) * d[1]) + (m0[2] + m1[2]) * d[2];
#pragma unroll
        for (int k = 0; k < 3; ++k) u[(1 + k) * vs + i] = m1[k];
        u[4 * vs + i] = e0 + T(0.5) * de;
    }
}

template <typename T>
static cudaError_t launch_gravity(int n, T* u, const T* phi, double dh, double dt, cudaStream_t st) {
    const size_t cells = (size_t)n * CELLS_PG;
    const size_t want = (cells + NT_GRAV - 1) / NT_GRAV;
    const unsigned grid = (unsigned)(want < (size_t)(1u << 30) ? want : (size_t)(1u << 30));
    k_gravity<T><<<grid, NT_GRAV, 0, st>>>(u, phi, n, (T)(dt / (2.0 * dh)));
    return cudaGetLastError();
}

}  // namespace gh

using namespace gh;

extern "C" int gamer_gravity_update(int precision, int n_groups, void* u, const void* phi, double dh, double dt,
                                    void* cuda_stream) {
    auto fail = [](int code, const char* msg) {
        set_thread_error(msg);
        return code;
    };
    if (precision != GAMER_FP32 && precision != GAMER_FP64) return fail(GAMER_ERR_ARG, "unknown precision");
    if (n_groups < 0) return fail(GAMER_ERR_ARG, "negative n_groups");
    if (!(dh > 0.0) || !(dt >= 0.0) || !std::isfinite(dh) || !std::isfinite(dt))
        return fail(GAMER_ERR_ARG, "dh must be positive and dt non-negative, both finite");
    if (n_groups == 0) return GAMER_OK;
    if (!u || !phi) return fail(GAMER_ERR_ARG, "u and phi are required");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = precision == GAMER_FP32
                        ? launch_gravity<float>(n_groups, static_cast<float*>(u), static_cast<const float*>(phi), dh,
                                                dt, st)
                        : launch_gravity<double>(n_groups, static_cast<double*>(u), static_cast<const double*>(phi),
                                                 dh, dt, st);
    if (e != cudaSuccess)
        return fail(GAMER_ERR_CUDA, (std::string("gravity launch: ") + cudaGetErrorString(e)).c_str());
    return GAMER_OK;
}
