// noalloc.cu -- gamer_hydro_diagnose_noalloc: the CFL time step and the
// conservation / positivity check without any device allocation.
//
// Who needs it: code that runs where cudaMalloc is not allowed or not
// wanted -- for example a host thread that must not synchronise the device
// (cudaMalloc and cudaFree can), a caller inside a memory pool or arena
// that owns every byte of the GPU, or a signal/timer callback that only
// wants a quick health check of the current state.  The regular
// gamer_hydro_diagnose needs a handle, and creating a handle allocates.
//
// How: the per-group partial results that the diagnostics kernels need as
// scratch live in one file-scope __device__ array of fixed size, shared by
// every call in the process.  Every call looks its address up on the
// current device with cudaGetSymbolAddress (host code may not use the
// array's name as a device pointer) and hands it to the kernels.  The
// address is not cached: after cudaDeviceReset, or when the primary
// context is released and created again, the module is loaded anew and an
// address kept from before would dangle.
#include <cmath>
#include <cstring>
#include <string>

#include "gamer_hydro.h"
#include "internal.h"

namespace gh {

// Largest number of patch groups (summed over levels) one call may cover.
constexpr int NOALLOC_MAX_GROUPS = 65536;

// Scratch layout inside the array, in bytes (each part 256-byte aligned):
// speed maxima [max groups] u64, sums [max groups][5] double, bad counts
// [max groups] int, per-level results [MAXLEV] DiagOut.
constexpr size_t NA_MAX_OFF = 0;
constexpr size_t NA_SUM_OFF = NA_MAX_OFF + sizeof(unsigned long long) * NOALLOC_MAX_GROUPS;
constexpr size_t NA_BAD_OFF = NA_SUM_OFF + sizeof(double) * NV * NOALLOC_MAX_GROUPS;
constexpr size_t NA_OUT_OFF = NA_BAD_OFF + sizeof(int) * NOALLOC_MAX_GROUPS;
constexpr size_t NA_BYTES = NA_OUT_OFF + ((sizeof(DiagOut) * MAXLEV + 255) / 256) * 256;
static_assert(NA_SUM_OFF % 256 == 0 && NA_BAD_OFF % 256 == 0 && NA_OUT_OFF % 256 == 0,
              "scratch parts must stay 256-byte aligned");

// 3.4 MB, held by every GPU that loads the library until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

namespace {

// Device address of the scratch array in the current device's context
// (the lookup allocates nothing).
cudaError_t scratch_address(unsigned char** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<unsigned char*>(p);
    return cudaSuccess;
}

template <typename T>
void fill_args(DiagArgs<T>& a, const gamer_hierarchy_t* H, double gamma, unsigned char* base) {
    memset(&a, 0, sizeof(a));
    int item = 0;
    for (int l = 0; l < H->n_levels; ++l) {
        a.lv[l].u = static_cast<const T*>(H->levels[l].u);
        a.lv[l].child = (l + 1 < H->n_levels) ? H->levels[l].child : nullptr;
        a.lv[l].n_groups = H->levels[l].n_groups;
        a.lv[l].item0 = item;
        item += H->levels[l].n_groups;
    }
    a.n_levels = H->n_levels;
    a.gamma = (T)gamma;
    a.gm1 = (T)(gamma - 1.0);
    a.pg_max = reinterpret_cast<unsigned long long*>(base + NA_MAX_OFF);
    a.pg_sum = reinterpret_cast<double*>(base + NA_SUM_OFF);
    a.pg_bad = reinterpret_cast<int*>(base + NA_BAD_OFF);
    a.out = reinterpret_cast<DiagOut*>(base + NA_OUT_OFF);
}

int fail(int code, const std::string& msg) {
    set_thread_error(msg);
    return code;
}

}  // namespace
}  // namespace gh

using namespace gh;

extern "C" int gamer_hydro_diagnose_noalloc(double gamma, int precision, const gamer_hierarchy_t* H,
                                            double cfl, void* cuda_stream, double* dt_out,
                                            double sums[5], int64_t* n_bad) {
    if (!(gamma > 1.0) || !std::isfinite(gamma)) return fail(GAMER_ERR_ARG, "gamma must be > 1");
    if (precision != GAMER_FP32 && precision != GAMER_FP64) return fail(GAMER_ERR_ARG, "unknown precision");
    if (!H || !H->levels) return fail(GAMER_ERR_ARG, "hierarchy is NULL");
    if (H->n_levels < 1 || H->n_levels > MAXLEV) return fail(GAMER_ERR_ARG, "n_levels must be in [1, 16]");
    if (dt_out && !(cfl > 0.0)) return fail(GAMER_ERR_ARG, "cfl must be positive");
    long long total = 0;
    for (int l = 0; l < H->n_levels; ++l) {
        const gamer_level_t& L = H->levels[l];
        if (L.n_groups < 0) return fail(GAMER_ERR_ARG, "negative n_groups");
        if (!(L.dh > 0.0)) return fail(GAMER_ERR_ARG, "dh must be positive");
        if (L.n_groups > 0 && !L.u) return fail(GAMER_ERR_ARG, "u is NULL on level " + std::to_string(l));
        if (L.n_groups > 0 && l + 1 < H->n_levels && !L.child)
            return fail(GAMER_ERR_ARG, "child map required below the finest level");
        total += L.n_groups;
    }
    if (total > NOALLOC_MAX_GROUPS)
        return fail(GAMER_ERR_ARG, "gamer_hydro_diagnose_noalloc covers at most " +
                                       std::to_string(NOALLOC_MAX_GROUPS) + " patch groups per call (got " +
                                       std::to_string(total) + ")");
    unsigned char* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return fail(GAMER_ERR_CUDA, std::string("scratch set-up: ") + cudaGetErrorString(e));
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // Every entry the kernels read (items [0, total), levels [0, n_levels))
    // is written earlier in the same call, so nothing has to be cleared.
    DiagOut out[MAXLEV];
    if (precision == GAMER_FP32) {
        DiagArgs<float> a;
        fill_args<float>(a, H, gamma, base);
        e = launch_diag<float>(a, (int)total, st);
    } else {
        DiagArgs<double> a;
        fill_args<double>(a, H, gamma, base);
        e = launch_diag<double>(a, (int)total, st);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, base + NA_OUT_OFF, sizeof(DiagOut) * H->n_levels, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(GAMER_ERR_CUDA, std::string("diagnostics: ") + cudaGetErrorString(e));
    if (dt_out) {
        double dt = INFINITY;
        for (int l = 0; l < H->n_levels; ++l) {
            if (H->levels[l].n_groups == 0) continue;
            double s;
            memcpy(&s, &out[l].smax_bits, sizeof(s));
            const double d = H->levels[l].dh / s;
            if (d < dt || d != d) dt = d;
        }
        *dt_out = cfl * dt;
    }
    if (sums) {
        for (int v = 0; v < NV; ++v) sums[v] = 0.0;
        for (int l = 0; l < H->n_levels; ++l) {
            const double dh = H->levels[l].dh, dV = dh * dh * dh;
            for (int v = 0; v < NV; ++v) sums[v] += out[l].sum[v] * dV;
        }
    }
    if (n_bad) {
        long long nb = 0;
        for (int l = 0; l < H->n_levels; ++l) nb += out[l].n_bad;
        *n_bad = nb;
    }
    return GAMER_OK;
}
