// step_reduce.cuh -- the end-of-step reduction shared by the stand-alone
// final kernel and by the last CTA of the fused FP32 sweep launch.
//
// Per level, the per-group diagnostics are combined in a fixed order
// (strided partials over NT_FIN threads, then a fixed tree), so the result
// does not depend on which kernel ran it.  dt follows Eq. CFL,
// dt = cfl * min_l dh_l / s_l in FP64, and the conserved sums are the leaf
// sums times dh^3, level by level.  With individual time steps level l
// takes 2^l steps per dt, so its bound on dt is cfl 2^l dh_l / s_l.
#pragma once
#include "common.cuh"

namespace gh {

constexpr int NT_FIN = 256;

// Result of one whole step, written on the device.
struct StepOut {
    double dt_used;     // dt of the step just taken
    double dt_next;     // dt the next step will use (held for a zyx step)
    double dt_cfl;      // Eq. CFL from the new state
    double sum[NV];     // leaf sums of u * dh^3
    long long n_bad;
    long long steps;
    long long status;   // nonzero: a dependency wait of the step gave up
};

struct LevelMeta {
    int item0[MAXLEV];
    int n[MAXLEV];
    double dh[MAXLEV];
    double dscale[MAXLEV];   // 1, or 2^l with individual time steps (level l takes 2^l steps per dt)
    int n_levels;
};

// Block-wide reduction.  Every thread of the block calls it (threads at or
// above NT_FIN only take part in the barriers).  Scratch: s_sum [NV][NT_FIN],
// s_max [NT_FIN], s_bad [NT_FIN] in shared memory.  The per-group inputs are
// read through L2 (they may have been written by other CTAs of the same
// launch).  The result goes to *out and, when out_host is given, to that
// mapped host copy as well (no copy node needed after the kernel).  status:
// the launch's wait-failure word, copied into the result and cleared.  *dt becomes the new value when update_dt is set (the next step
// is an xyz step), otherwise it is held (one dt for a forward and backward
// sweep set, Sec. 2.2).  Products are rounded explicitly so that the result
// is the same under any contraction setting of the including file.
__device__ __forceinline__ void step_reduce(const LevelMeta& m, const unsigned long long* pg_max,
                                            const double* pg_sum, const int* pg_bad, double cfl, double* dt,
                                            int update_dt, StepOut* out, StepOut* out_host, unsigned* status,
                                            double* s_sum, unsigned long long* s_max, long long* s_bad) {
    const int t = threadIdx.x;
    const bool act = t < NT_FIN;
    double tot[NV] = {0, 0, 0, 0, 0};
    double dtc = INFINITY;
    long long nb = 0;
    const double dt_used = *dt;
    for (int l = 0; l < m.n_levels; ++l) {
        if (act) {
            double sum[NV] = {0, 0, 0, 0, 0};
            unsigned long long mx = 0ull;
            long long bad = 0;
            for (int i = t; i < m.n[l]; i += NT_FIN) {
                const int it = m.item0[l] + i;
#pragma unroll
                for (int v = 0; v < NV; ++v) sum[v] += __ldcg(pg_sum + (size_t)it * NV + v);
                mx = max(mx, __ldcg(pg_max + it));
                bad += __ldcg(pg_bad + it);
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) s_sum[v * NT_FIN + t] = sum[v];
            s_max[t] = mx;
            s_bad[t] = bad;
        }
        __syncthreads();
        for (int w = NT_FIN / 2; w > 0; w >>= 1) {
            if (t < w) {
#pragma unroll
                for (int v = 0; v < NV; ++v) s_sum[v * NT_FIN + t] += s_sum[v * NT_FIN + t + w];
                s_max[t] = max(s_max[t], s_max[t + w]);
                s_bad[t] += s_bad[t + w];
            }
            __syncthreads();
        }
        if (t == 0 && m.n[l] > 0) {
            const double dV = __dmul_rn(__dmul_rn(m.dh[l], m.dh[l]), m.dh[l]);
#pragma unroll
            for (int v = 0; v < NV; ++v) tot[v] = __dadd_rn(tot[v], __dmul_rn(s_sum[v * NT_FIN], dV));
            const double s = __longlong_as_double((long long)s_max[0]);
            const double d = (m.dh[l] * m.dscale[l]) / s;
            if (d < dtc || d != d) dtc = d;
            nb += s_bad[0];
        }
        __syncthreads();
    }
    if (t == 0) {
        const double dnew = cfl * dtc;
        StepOut o;
        o.dt_used = dt_used;
        o.dt_cfl = dnew;
        o.dt_next = update_dt ? dnew : dt_used;
#pragma unroll
        for (int v = 0; v < NV; ++v) o.sum[v] = tot[v];
        o.n_bad = nb;
        o.steps = out->steps + 1;
        o.status = 0;
        if (status != nullptr) {
            o.status = *status;
            *status = 0u;
        }
        *out = o;
        if (out_host != nullptr) *out_host = o;
        if (update_dt) *dt = dnew;
    }
}

}  // namespace gh
