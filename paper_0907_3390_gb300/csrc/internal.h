// internal.h -- declarations shared between the kernel files and the C-ABI
// host code (not part of the public interface).
#pragma once
#include <cstddef>
#include <cstdint>
#include <string>
#include <cuda_runtime.h>

#include "common.cuh"
#include "step_reduce.cuh"

namespace gh {

// ---- sweep kernels
// variant 0: pipelined (512 threads); 1: non-pipelined (256 or 512 threads)
cudaError_t launch_sweep_f32(const SweepArgs<float>& a, int order, int lim, int variant, int threads, int grid,
                             cudaStream_t st);
size_t sweep_f32_smem();
// xyz + zyx pair of one level (a.pair set, a.total = 2 n, lv[1] = lv[0] with u / u_out swapped)
cudaError_t launch_sweep_pair(const SweepArgs<float>& a, int lim, int grid, cudaStream_t st);
cudaError_t sweep_f32_init();
// threads per block: 128 or 256
cudaError_t launch_pg_f64(const LevelArgs<double>& L, int g0, int count, int order, int lim,
                          double gamma, double gm1, const double* dt, double* stage, int threads,
                          cudaStream_t st);
size_t stage_f64_bytes_per_group();

// ---- fix-up: coarse level c corrected from fine level c+1
template <typename T>
struct FixArgs {
    const int* list;      // coarse patches to visit
    T* uc;                // coarse u_out
    const T* uf;          // fine u_out
    const int* nbr;       // coarse map
    const int* child;     // coarse child map
    const T* flux_c;      // coarse face fluxes
    const T* flux_f;      // fine face fluxes (of the finer level's first step)
    const T* flux_f2;     // fine face fluxes of its second step (individual time steps), or nullptr
    int n_c, n_f;         // groups on the two levels
    const double* dt;     // device slot holding the time step
    double dh;            // coarse cell width
    double dts;           // the coarse level's share of the device dt (1 or 2^-l)
};
template <typename T>
cudaError_t launch_fixup(const FixArgs<T>& a, int n_list, cudaStream_t st);

// ---- rebuild of the refinement map (regrid.cu)
template <typename T>
struct FlagArgs {
    const T* u;           // the level's state
    const int* nbr;       // its map
    int n_groups;
    int criterion;        // 0 density gradient, 1 pressure gradient, 2 density threshold
    double threshold;
    int n_buffer;         // flag buffer in cells, 0..8
    double gamma;
    unsigned* masks;      // [8 n_groups] output
};
template <typename T>
cudaError_t launch_flag(const FlagArgs<T>& a, cudaStream_t st);

template <typename T>
struct PrepArgs {
    const T* phi_c;       // coarser level's potential [8 n_c][8][8][8]
    const int* nbrc;      // coarser level's map
    int n_c;              // coarser level's groups
    const int* parent;    // [n] parent patch (on the coarser level) of every group
    const T* u;           // the level's state (density = variable 0)
    int n;                // the level's groups
    T* phi_blk;           // [n][18][18][18] output
    T* rho_blk;           // [n][16][16][16] output
};
template <typename T>
cudaError_t launch_poisson_prepare(const PrepArgs<T>& a, cudaStream_t st);

template <typename T>
struct RefineArgs {
    const T* uc;          // parent level's state
    const int* nbrc;      // parent level's map
    int n_c;              // parent level's groups
    const int* parent_new;// [n_new] parent patch of every new group
    const int* inherit;   // [n_new] old group to copy, or -1: interpolate
    const T* u_old;       // previous state of the rebuilt level (n_old groups), or nullptr
    int n_old;
    T* u_new;             // [5][8 n_new][512] output
    int n_new;
};
template <typename T>
cudaError_t launch_refine(const RefineArgs<T>& a, cudaStream_t st);

// ---- diagnostics
template <typename T>
struct DiagLevel {
    const T* u;
    const int* child;
    int n_groups;
    int item0;
};
struct DiagOut {
    unsigned long long smax_bits;  // bit pattern of the largest signal speed
    double sum[NV];                // leaf sums of u (not yet times dV)
    long long n_bad;
};
template <typename T>
struct DiagArgs {
    DiagLevel<T> lv[MAXLEV];
    int n_levels;
    T gamma, gm1;
    unsigned long long* pg_max;   // [total]
    double* pg_sum;               // [total][5]
    int* pg_bad;                  // [total]
    DiagOut* out;                 // [n_levels]
};
template <typename T>
cudaError_t launch_diag(const DiagArgs<T>& a, int total, cudaStream_t st);
// per-group diagnostics only (no per-level reduction)
template <typename T>
cudaError_t launch_diag_groups(const DiagArgs<T>& a, int total, cudaStream_t st);

// One block: per-level reduction of the per-group diagnostics in fixed
// order, then dt from Eq. CFL (written to *dt when update_dt != 0).
cudaError_t launch_step_final(const DiagArgs<float>& a32, const DiagArgs<double>& a64, bool fp64,
                              const double* dh, const double* dscale, double cfl, double* dt, int update_dt,
                              StepOut* out, StepOut* out_host, cudaStream_t st);
cudaError_t launch_set_dt(double* slot, double dt, cudaStream_t st);

// Message of the last failed handle-free call on this thread (read back by
// gamer_hydro_last_error(NULL)).
void set_thread_error(const std::string& msg);

}  // namespace gh
