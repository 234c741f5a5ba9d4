// hydro_api.cu -- the C ABI of include/gamer_hydro.h: handle, validation of
// hierarchy snapshots, scratch management, launch sequencing, CUDA-graph
// replay of whole steps, and error reporting.
#include <algorithm>
#include <cstdint>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "gamer_hydro.h"
#include "internal.h"

using namespace gh;

namespace {

thread_local std::string g_create_error;

}  // namespace

void gh::set_thread_error(const std::string& msg) { g_create_error = msg; }

namespace {

struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    uint64_t last_use = 0;
};

struct LevelCache {
    int n_groups = 0;
    double dh = 0.0;
    std::vector<int> fix_list;    // coarse patches visited by the fix-up of this level
    int* d_fix_list = nullptr;
    void* own_flux = nullptr;     // handle-owned face fluxes when the caller gives none
    void* own_flux2 = nullptr;    // fluxes of a level's second step (individual time steps)
    void* ghost = nullptr;        // FP32 coarse-fine ghost slots (levels above 0)
    int* d_gslot = nullptr;       // [n_groups] slot of a group, -1 without a coarse region
    int* d_slot_g = nullptr;      // [n_slots] group of each slot
    int n_slots = 0;
    unsigned* d_fneed = nullptr;  // [n_groups] face-flux columns the fix-ups read (FP32, own fluxes)
};

}  // namespace

struct gamer_hydro_s {
    double gamma = 5.0 / 3.0;
    int limiter = GAMER_LIMITER_VANLEER;
    int precision = GAMER_FP32;
    int device = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    int parity[32] = {0};
    std::string err;

    // hierarchy cache (maps are validated once per version)
    bool have_version = false;
    uint64_t version = 0;
    int n_levels = 0;
    std::vector<LevelCache> lv;
    int total_groups = 0;

    // scratch
    int* d_queue = nullptr;       // [4]: work queue, finished CTAs, pair launch counter, pair status
    unsigned* d_ready = nullptr;  // [pair_n] publication marks of pair launches
    int* d_order1 = nullptr;      // [pair_n] zyx work order of pair launches
    int pair_n = 0;
    int hold = -1;                // group whose mark the next pair launch withholds (test hook)
    unsigned long long* d_pg_max = nullptr;
    double* d_pg_sum = nullptr;
    int* d_pg_bad = nullptr;
    DiagOut* d_out = nullptr;
    DiagOut* h_out = nullptr;     // pinned
    int diag_cap = 0;
    double* d_stage = nullptr;
    int stage_groups = 0;

    // launch configuration (gamer_hydro_tune may change it)
    int f32_variant = 0;          // 0 pipelined, 1 non-pipelined
    int sweep_threads = 512;
    int grid_mode = 0;            // 0: one CTA per SM (capped by items); 1: balanced rounds
    int f64_threads = 256;
    int f64_chunk = 2048;
    bool tuned = false;
    int individual = 0;           // individual time steps per level (gamer_hydro_set_time_steps)

    // whole steps (gamer_hydro_step): captured CUDA graphs keyed by the
    // launch arguments, replayed on the handle's stream
    std::map<std::string, GraphEntry> graphs;
    uint64_t use_clock = 0;
    cudaStream_t cap_stream = nullptr;
    double* d_dt = nullptr;       // device time step read by every kernel
    bool dt_ready = false;        // d_dt holds the step dt of the current state
    uint64_t dt_version = 0;
    StepOut* d_step = nullptr;    // device result of the last step
    StepOut* h_step = nullptr;    // mapped pinned host copy, written by the step's last kernel
    StepOut* h_step_dev = nullptr;// the same memory as the device addresses it
    cudaEvent_t step_event = nullptr;
    cudaEvent_t prof_ev[2] = {nullptr, nullptr};   // recorded around the sweep launch
};

namespace {

int fail(gamer_hydro_t h, int code, const std::string& msg) {
    if (h) h->err = msg;
    else g_create_error = msg;
    return code;
}

int cuda_fail(gamer_hydro_t h, cudaError_t e, const char* what) {
    return fail(h, GAMER_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(h, call)                                                   \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);      \
    } while (0)

int floordiv(int a, int b) {
    int q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}

// Host mirror of the device region resolution: source group of a position
// (in patch units relative to group g) after the outflow clamp.  Returns
// the group index (>= 0), -1 (coarse) or another negative map value.
int resolve_patch(const std::vector<int>& nbr, int g, int q[3]) {
    int o[3];
    for (int a = 0; a < 3; ++a) {
        o[a] = floordiv(q[a], 2);
        if (o[a] != 0) {
            int e[3] = {0, 0, 0};
            e[a] = o[a];
            if (nbr[(size_t)g * 26 + dir_index(e[0], e[1], e[2])] == -2) {
                q[a] = q[a] < 0 ? 0 : 1;
                o[a] = 0;
            }
        }
    }
    for (int a = 0; a < 3; ++a) q[a] -= 2 * o[a];
    if (!(o[0] | o[1] | o[2])) return g;
    return nbr[(size_t)g * 26 + dir_index(o[0], o[1], o[2])];
}

template <typename T>
void fill_level(LevelArgs<T>& a, const gamer_level_t* L, int l, const gamer_hydro_s* h) {
    const gamer_level_t& c = L[l];
    a.u = static_cast<const T*>(c.u);
    a.u_out = static_cast<T*>(c.u_out);
    a.nbr = c.nbr;
    a.flux = static_cast<T*>(c.face_flux ? c.face_flux : h->lv[l].own_flux);
    if (h->n_levels == 1) a.flux = nullptr;
    // a caller's flux buffer gets every plane; the handle's own only what the fix-ups read
    a.fneed = (c.face_flux == nullptr && h->precision == GAMER_FP32) ? h->lv[l].d_fneed : nullptr;
    a.parent = l > 0 ? c.parent : nullptr;
    a.uc = l > 0 ? static_cast<const T*>(L[l - 1].u) : nullptr;
    a.nbrc = l > 0 ? L[l - 1].nbr : nullptr;
    a.ghost = nullptr;
    a.gslot = nullptr;
    a.slot_g = nullptr;
    a.n_slots = 0;
    if (l > 0 && h->precision == GAMER_FP32) {
        a.ghost = static_cast<T*>(h->lv[l].ghost);
        a.gslot = h->lv[l].d_gslot;
        a.slot_g = h->lv[l].d_slot_g;
        a.n_slots = h->lv[l].n_slots;
    }
    a.n_groups = c.n_groups;
    a.n_groups_c = l > 0 ? L[l - 1].n_groups : 0;
    a.item0 = 0;
    a.dh = c.dh;
    a.ucn = nullptr;
    a.dts = 1.0;
    a.cw = 0.0;
}

size_t elem_size(const gamer_hydro_s* h) { return h->precision == GAMER_FP64 ? 8 : 4; }

int ensure_diag(gamer_hydro_t h, int total) {
    if (total <= h->diag_cap && h->d_out) return GAMER_OK;
    cudaFree(h->d_pg_max);
    cudaFree(h->d_pg_sum);
    cudaFree(h->d_pg_bad);
    h->d_pg_max = nullptr; h->d_pg_sum = nullptr; h->d_pg_bad = nullptr;
    int cap = std::max(total, 1);
    CK(h, cudaMalloc(&h->d_pg_max, sizeof(unsigned long long) * cap));
    CK(h, cudaMalloc(&h->d_pg_sum, sizeof(double) * NV * cap));
    CK(h, cudaMalloc(&h->d_pg_bad, sizeof(int) * cap));
    if (!h->d_out) {
        CK(h, cudaMalloc(&h->d_out, sizeof(DiagOut) * MAXLEV));
        CK(h, cudaMallocHost(&h->h_out, sizeof(DiagOut) * MAXLEV));
    }
    h->diag_cap = cap;
    return GAMER_OK;
}

void drop_graphs(gamer_hydro_t h) {
    for (auto& kv : h->graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    h->graphs.clear();
}

void drop_hierarchy(gamer_hydro_t h) {
    for (auto& c : h->lv) {
        cudaFree(c.d_fix_list);
        cudaFree(c.own_flux);
        cudaFree(c.own_flux2);
        cudaFree(c.ghost);
        cudaFree(c.d_gslot);
        cudaFree(c.d_slot_g);
        cudaFree(c.d_fneed);
    }
    h->lv.clear();
    h->have_version = false;
    drop_graphs(h);
}

// Source of ghost region r = (oz+1)*9 + (oy+1)*3 + (ox+1) of group g: the
// same-level group after the outflow clamp (axes whose face neighbour is -2
// fold into the group), -1 for a region on the coarser level, -2 outside.
int region_source(const std::vector<int>& nbr, int g, int r) {
    int o[3] = {r % 3 - 1, (r / 3) % 3 - 1, r / 9 - 1};
    for (int a = 0; a < 3; ++a) {
        if (o[a] == 0) continue;
        int e[3] = {0, 0, 0};
        e[a] = o[a];
        if (nbr[(size_t)g * 26 + dir_index(e[0], e[1], e[2])] == -2) o[a] = 0;
    }
    return (o[0] | o[1] | o[2]) ? nbr[(size_t)g * 26 + dir_index(o[0], o[1], o[2])] : g;
}

// Validate a hierarchy snapshot (once per version) and build the fix-up
// work lists.  Maps are copied to the host; this synchronises the device.
int prepare(gamer_hydro_t h, const gamer_hierarchy_t* H) {
    if (!H || !H->levels) return fail(h, GAMER_ERR_ARG, "hierarchy is NULL");
    if (H->n_levels < 1 || H->n_levels > MAXLEV)
        return fail(h, GAMER_ERR_ARG, "n_levels must be in [1, 16]");
    if (h->have_version && h->version == H->version && h->n_levels == H->n_levels) {
        for (int l = 0; l < H->n_levels; ++l)
            if (H->levels[l].n_groups != h->lv[l].n_groups || H->levels[l].dh != h->lv[l].dh)
                return fail(h, GAMER_ERR_STATE, "maps changed without a new hierarchy version");
        return GAMER_OK;
    }
    drop_hierarchy(h);
    const int n = H->n_levels;
    std::vector<std::vector<int>> nbr(n), parent(n), child(n);
    int total = 0;
    for (int l = 0; l < n; ++l) {
        const gamer_level_t& L = H->levels[l];
        if (L.n_groups < 0) return fail(h, GAMER_ERR_ARG, "negative n_groups");
        if (!(L.dh > 0.0)) return fail(h, GAMER_ERR_ARG, "dh must be positive");
        if (L.n_groups > 0 && (!L.u || !L.u_out || !L.nbr))
            return fail(h, GAMER_ERR_ARG, "u, u_out and nbr are required");
        if (L.n_groups > 0 && L.u == L.u_out)
            return fail(h, GAMER_ERR_ARG, "u_out must not alias u");
        total += L.n_groups;
        nbr[l].resize((size_t)L.n_groups * 26);
        if (L.n_groups > 0)
            CK(h, cudaMemcpy(nbr[l].data(), L.nbr, sizeof(int) * nbr[l].size(), cudaMemcpyDeviceToHost));
        if (l > 0 && L.n_groups > 0) {
            if (!L.parent) return fail(h, GAMER_ERR_MAP, "parent map required above level 0");
            parent[l].resize(L.n_groups);
            CK(h, cudaMemcpy(parent[l].data(), L.parent, sizeof(int) * L.n_groups, cudaMemcpyDeviceToHost));
        }
        if (l + 1 < n && L.n_groups > 0) {
            if (!L.child) return fail(h, GAMER_ERR_MAP, "child map required below the finest level");
            child[l].resize((size_t)8 * L.n_groups);
            CK(h, cudaMemcpy(child[l].data(), L.child, sizeof(int) * child[l].size(), cudaMemcpyDeviceToHost));
        }
    }
    for (int l = 0; l < n; ++l) {
        const int ng = H->levels[l].n_groups;
        for (int v : nbr[l]) {
            if (v >= ng || v < -2) return fail(h, GAMER_ERR_MAP, "nbr entry out of range on level " + std::to_string(l));
            if (v == -1 && l == 0) return fail(h, GAMER_ERR_MAP, "coarse (-1) neighbour on level 0");
        }
        // every ghost region must resolve (after the outflow clamp) to a
        // same-level group, or to the coarser level above level 0
        for (int g = 0; g < ng; ++g)
            for (int r = 0; r < 27; ++r) {
                if (r == 13) continue;
                const int src = region_source(nbr[l], g, r);
                if (src >= 0 || (src == -1 && l > 0)) continue;
                return fail(h, GAMER_ERR_MAP, "ghost region of group " + std::to_string(g) + " on level " +
                                                  std::to_string(l) + " does not resolve");
            }
        if (l > 0) {
            const int nc = H->levels[l - 1].n_groups;
            for (int g = 0; g < ng; ++g) {
                int P = parent[l][g];
                if (P < 0 || P >= 8 * nc) return fail(h, GAMER_ERR_MAP, "parent out of range on level " + std::to_string(l));
                if (child[l - 1][P] != g) return fail(h, GAMER_ERR_MAP, "child[parent[g]] != g on level " + std::to_string(l));
                // proper nesting: the 26 neighbours of the parent patch exist
                bool needs = false;
                for (int d = 0; d < 26; ++d) needs |= nbr[l][(size_t)g * 26 + d] == -1;
                if (!needs) continue;
                const int gc = P >> 3, lp = P & 7;
                for (int dz = -1; dz <= 1; ++dz)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            int q[3] = {(lp & 1) + dx, ((lp >> 1) & 1) + dy, ((lp >> 2) & 1) + dz};
                            if (resolve_patch(nbr[l - 1], gc, q) < 0)
                                return fail(h, GAMER_ERR_MAP, "proper nesting violated on level " + std::to_string(l));
                        }
            }
        }
        if (l + 1 < n) {
            const int nf = H->levels[l + 1].n_groups;
            for (int c : child[l])
                if (c < -1 || c >= nf) return fail(h, GAMER_ERR_MAP, "child entry out of range on level " + std::to_string(l));
        }
    }
    h->lv.assign(n, LevelCache());
    for (int l = 0; l < n; ++l) {
        LevelCache& c = h->lv[l];
        c.n_groups = H->levels[l].n_groups;
        c.dh = H->levels[l].dh;
        if (n > 1 && !H->levels[l].face_flux && c.n_groups > 0)
            CK(h, cudaMalloc(&c.own_flux, (size_t)c.n_groups * FLUX_PG * elem_size(h)));
        if (n > 1 && h->individual && c.n_groups > 0)
            CK(h, cudaMalloc(&c.own_flux2, (size_t)c.n_groups * FLUX_PG * elem_size(h)));
        if (l > 0 && h->precision == GAMER_FP32 && c.n_groups > 0) {
            // a slot for every group with a ghost region on the coarser level
            std::vector<int> slot(c.n_groups, -1), slot_g;
            for (int g = 0; g < c.n_groups; ++g)
                for (int r = 0; r < 27 && slot[g] < 0; ++r)
                    if (r != 13 && region_source(nbr[l], g, r) == -1) {
                        slot[g] = (int)slot_g.size();
                        slot_g.push_back(g);
                    }
            c.n_slots = (int)slot_g.size();
            CK(h, cudaMalloc(&c.d_gslot, sizeof(int) * c.n_groups));
            CK(h, cudaMemcpy(c.d_gslot, slot.data(), sizeof(int) * c.n_groups, cudaMemcpyHostToDevice));
            if (c.n_slots > 0) {
                CK(h, cudaMalloc(&c.ghost, (size_t)c.n_slots * GHOST_PG * sizeof(float)));
                CK(h, cudaMalloc(&c.d_slot_g, sizeof(int) * c.n_slots));
                CK(h, cudaMemcpy(c.d_slot_g, slot_g.data(), sizeof(int) * c.n_slots, cudaMemcpyHostToDevice));
            }
        }
        if (l + 1 < n) {
            for (int P = 0; P < 8 * c.n_groups; ++P) {
                bool take = child[l][P] >= 0;
                if (!take) {
                    const int g = P >> 3, lp = P & 7;
                    for (int ax = 0; ax < 3 && !take; ++ax)
                        for (int s = -1; s <= 1 && !take; s += 2) {
                            int q[3] = {lp & 1, (lp >> 1) & 1, (lp >> 2) & 1};
                            q[ax] += s;
                            int gq = g;
                            if (q[ax] < 0 || q[ax] > 1) {
                                int e[3] = {0, 0, 0};
                                e[ax] = s;
                                gq = nbr[l][(size_t)g * 26 + dir_index(e[0], e[1], e[2])];
                                q[ax] = q[ax] < 0 ? 1 : 0;
                            }
                            if (gq >= 0 && child[l][8 * gq + (q[2] * 2 + q[1]) * 2 + q[0]] >= 0) take = true;
                        }
                }
                if (take) c.fix_list.push_back(P);
            }
            if (!c.fix_list.empty()) {
                CK(h, cudaMalloc(&c.d_fix_list, sizeof(int) * c.fix_list.size()));
                CK(h, cudaMemcpy(c.d_fix_list, c.fix_list.data(), sizeof(int) * c.fix_list.size(),
                                 cudaMemcpyHostToDevice));
            }
        }
    }
    // Face fluxes the fix-ups read (k_fixup), per group as bit 4 ax + q for
    // the sweep columns along axis ax in transverse quarter q (q = 2 p_t2 +
    // p_t1 over the patch positions along the transverse axes t1 < t2): a
    // leaf patch's face towards a refined same-level patch (coarse side),
    // and the whole face of the refined patch's child group towards it
    // (fine side).
    if (n > 1 && h->precision == GAMER_FP32) {
        std::vector<std::vector<unsigned>> need(n);
        for (int l = 0; l < n; ++l) need[l].assign(H->levels[l].n_groups, 0u);
        for (int l = 0; l + 1 < n; ++l)
            for (int P = 0; P < 8 * H->levels[l].n_groups; ++P) {
                if (child[l][P] >= 0) continue;
                const int g = P >> 3, lp = P & 7;
                const int pc[3] = {lp & 1, (lp >> 1) & 1, (lp >> 2) & 1};
                for (int ax = 0; ax < 3; ++ax)
                    for (int s = -1; s <= 1; s += 2) {
                        int q[3] = {pc[0], pc[1], pc[2]};
                        q[ax] += s;
                        const int gq = resolve_patch(nbr[l], g, q);
                        if (gq < 0) continue;
                        const int fq = child[l][8 * gq + (q[2] * 2 + q[1]) * 2 + q[0]];
                        if (fq < 0) continue;
                        const int t1 = ax == 0 ? 1 : 0, t2 = ax == 2 ? 1 : 2;
                        need[l][g] |= 1u << (4 * ax + 2 * pc[t2] + pc[t1]);
                        need[l + 1][fq] |= 0xFu << (4 * ax);
                    }
            }
        for (int l = 0; l < n; ++l) {
            LevelCache& c = h->lv[l];
            if (c.n_groups == 0) continue;
            CK(h, cudaMalloc(&c.d_fneed, sizeof(unsigned) * c.n_groups));
            CK(h, cudaMemcpy(c.d_fneed, need[l].data(), sizeof(unsigned) * c.n_groups, cudaMemcpyHostToDevice));
        }
    }
    // A pair launch writes a group's zyx result over its input once the xyz
    // sets of the group's 26 neighbours are done, which covers every reader
    // of that input only if the neighbour relation is symmetric.
    bool symmetric = n == 1;
    for (int g = 0; symmetric && g < total; ++g)
        for (int d = 0; d < 26 && symmetric; ++d) {
            const int q = nbr[0][(size_t)g * 26 + d];
            const int dd = d < 13 ? d : d + 1;               // 27-cell index of direction d
            const int opp = 26 - dd;                          // the opposite direction
            if (q >= 0 && nbr[0][(size_t)q * 26 + (opp < 13 ? opp : opp - 1)] != g) symmetric = false;
        }
    if (!symmetric && h->pair_n) {
        cudaFree(h->d_ready);
        cudaFree(h->d_order1);
        h->d_ready = nullptr;
        h->d_order1 = nullptr;
        h->pair_n = 0;
    }
    if (n == 1 && symmetric && h->precision == GAMER_FP32 && total > 0) {
        // zyx work order of pair launches: a group's zyx set needs the xyz
        // results of the group and of its 26 neighbours, and xyz items are
        // taken in index order, so the zyx items go by the last of those
        // indices (ties by group)
        const int ng = total;
        std::vector<std::pair<int, int>> key(ng);
        for (int g = 0; g < ng; ++g) {
            int k = g;
            for (int d = 0; d < 26; ++d) k = std::max(k, nbr[0][(size_t)g * 26 + d]);
            key[g] = {k, g};
        }
        std::sort(key.begin(), key.end());
        std::vector<int> order(ng);
        for (int i = 0; i < ng; ++i) order[i] = key[i].second;
        if (h->pair_n != ng) {
            cudaFree(h->d_ready);
            cudaFree(h->d_order1);
            h->d_ready = nullptr;
            h->d_order1 = nullptr;
            h->pair_n = 0;
            CK(h, cudaMalloc(&h->d_ready, sizeof(unsigned) * ng));
            CK(h, cudaMemset(h->d_ready, 0, sizeof(unsigned) * ng));   // below every launch's mark
            CK(h, cudaMalloc(&h->d_order1, sizeof(int) * ng));
            h->pair_n = ng;
        }
        CK(h, cudaMemcpy(h->d_order1, order.data(), sizeof(int) * ng, cudaMemcpyHostToDevice));
    }
    h->n_levels = n;
    h->total_groups = total;
    h->version = H->version;
    h->have_version = true;
    if (h->precision == GAMER_FP64) {
        // staging blocks of the plain FP64 path, allocated here so that no
        // allocation happens while a step is being captured
        int need = 0;
        for (int l = 0; l < n; ++l) need = std::max(need, std::min(h->f64_chunk, H->levels[l].n_groups));
        if (h->stage_groups < need) {
            cudaFree(h->d_stage);
            h->d_stage = nullptr;
            CK(h, cudaMalloc(&h->d_stage, stage_f64_bytes_per_group() * need));
            h->stage_groups = need;
        }
    }
    return ensure_diag(h, total);
}

// Per-call pointer checks (u / u_out may change on every call).
int check_pointers(gamer_hydro_t h, const gamer_hierarchy_t* H, bool need_out) {
    for (int l = 0; l < H->n_levels; ++l) {
        const gamer_level_t& L = H->levels[l];
        if (L.n_groups == 0) continue;
        if (!L.u || !L.nbr) return fail(h, GAMER_ERR_ARG, "u and nbr are required on level " + std::to_string(l));
        if (need_out && !L.u_out) return fail(h, GAMER_ERR_ARG, "u_out is NULL on level " + std::to_string(l));
        if (need_out && L.u == L.u_out) return fail(h, GAMER_ERR_ARG, "u_out must not alias u");
        // the FP32 kernels move 16-byte quads of patch rows
        if ((reinterpret_cast<uintptr_t>(L.u) | (need_out ? reinterpret_cast<uintptr_t>(L.u_out) : 0)) & 15)
            return fail(h, GAMER_ERR_ARG, "u and u_out must be 16-byte aligned");
    }
    return GAMER_OK;
}

// Persistent-kernel grid: one CTA per SM, capped by the number of items;
// the balanced mode keeps the same number of rounds with fewer CTAs.
int sweep_grid(const gamer_hydro_s* h, int items) {
    int g = std::min(items, h->sm_count);
    if (h->grid_mode == 1 && g > 0) {
        const int rounds = (items + g - 1) / g;
        g = (items + rounds - 1) / rounds;
    }
    return std::max(g, 1);
}

int check_level_arg(gamer_hydro_t h, const gamer_hierarchy_t* H, int level) {
    if (level < 0 || level >= H->n_levels) return fail(h, GAMER_ERR_ARG, "level out of range");
    return GAMER_OK;
}

// Sweep set of level l reading dt from h->d_dt; `diag` fuses the
// diagnostics of the new state into the FP32 launch (single level only).
// Per-call options of one level's sweep set (individual time steps): the
// coarser level's state after its sweep set and the time weight of the
// coarse ghosts, this level's share of the device dt, the face-flux buffer
// to write.
struct LevelStep {
    const void* ucn = nullptr;
    double cw = 0.0;
    double dts = 1.0;
    void* flux = nullptr;
};

template <typename T>
void apply_step(LevelArgs<T>& a, const LevelStep* ls) {
    if (!ls) return;
    a.ucn = static_cast<const T*>(ls->ucn);
    a.cw = ls->cw;
    a.dts = ls->dts;
    if (ls->flux) a.flux = static_cast<T*>(ls->flux);
}

int advance_level_impl(gamer_hydro_t h, const gamer_hierarchy_t* H, int l, int order,
                       const LevelStep* ls = nullptr) {
    const gamer_level_t* L = H->levels;
    if (L[l].n_groups == 0) return GAMER_OK;
    if (h->precision == GAMER_FP32) {
        SweepArgs<float> a;
        memset(&a, 0, sizeof(a));
        fill_level<float>(a.lv[0], L, l, h);
        apply_step(a.lv[0], ls);
        a.n_levels = 1;
        a.total = L[l].n_groups;
        a.queue = h->d_queue;
        a.done = reinterpret_cast<unsigned*>(h->d_queue + 1);
        a.dt = h->d_dt;
        a.gamma = (float)h->gamma;
        a.gm1 = (float)(h->gamma - 1.0);
        CK(h, launch_sweep_f32(a, order, h->limiter, h->f32_variant, h->sweep_threads, sweep_grid(h, a.total),
                               h->stream));
    } else {
        LevelArgs<double> a;
        memset(&a, 0, sizeof(a));
        fill_level<double>(a, L, l, h);
        apply_step(a, ls);
        const int chunk = std::min(h->f64_chunk, L[l].n_groups);
        if (h->stage_groups < chunk) {
            cudaFree(h->d_stage);
            h->d_stage = nullptr;
            CK(h, cudaMalloc(&h->d_stage, stage_f64_bytes_per_group() * chunk));
            h->stage_groups = chunk;
        }
        for (int g0 = 0; g0 < L[l].n_groups; g0 += chunk) {
            const int cnt = std::min(chunk, L[l].n_groups - g0);
            CK(h, launch_pg_f64(a, g0, cnt, order, h->limiter, h->gamma, h->gamma - 1.0, h->d_dt,
                                h->d_stage, h->f64_threads, h->stream));
        }
    }
    return GAMER_OK;
}

// Per-call options of a fix-up (individual time steps): the coarse fluxes
// of this coarse step, the finer fluxes of its two steps, the finer state
// (after its two steps), the coarse level's share of the device dt.
struct FixStep {
    const void* fc = nullptr;
    const void* ff = nullptr;
    const void* ff2 = nullptr;
    const void* uf = nullptr;
    double dts = 1.0;
};

int fixup_impl(gamer_hydro_t h, const gamer_hierarchy_t* H, int l, const FixStep* fs = nullptr) {
    const gamer_level_t* L = H->levels;
    const LevelCache& c = h->lv[l];
    if (c.fix_list.empty()) return GAMER_OK;
    const void* fc = L[l].face_flux ? L[l].face_flux : h->lv[l].own_flux;
    const void* ff = L[l + 1].face_flux ? L[l + 1].face_flux : h->lv[l + 1].own_flux;
    const void* ff2 = nullptr;
    const void* uf = L[l + 1].u_out;
    double dts = 1.0;
    if (fs) {
        fc = fs->fc;
        ff = fs->ff;
        ff2 = fs->ff2;
        uf = fs->uf;
        dts = fs->dts;
    }
    if (h->precision == GAMER_FP32) {
        FixArgs<float> a{c.d_fix_list, (float*)L[l].u_out, (const float*)uf, L[l].nbr,
                         L[l].child, (const float*)fc, (const float*)ff, (const float*)ff2, L[l].n_groups,
                         L[l + 1].n_groups, h->d_dt, L[l].dh, dts};
        CK(h, launch_fixup<float>(a, (int)c.fix_list.size(), h->stream));
    } else {
        FixArgs<double> a{c.d_fix_list, (double*)L[l].u_out, (const double*)uf, L[l].nbr,
                          L[l].child, (const double*)fc, (const double*)ff, (const double*)ff2, L[l].n_groups,
                          L[l + 1].n_groups, h->d_dt, L[l].dh, dts};
        CK(h, launch_fixup<double>(a, (int)c.fix_list.size(), h->stream));
    }
    return GAMER_OK;
}

template <typename T>
void diag_args(gamer_hydro_t h, const gamer_hierarchy_t* H, DiagArgs<T>& a) {
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
    a.gamma = (T)h->gamma;
    a.gm1 = (T)(h->gamma - 1.0);
    a.pg_max = h->d_pg_max;
    a.pg_sum = h->d_pg_sum;
    a.pg_bad = h->d_pg_bad;
    a.out = h->d_out;
}

template <typename T>
int diag_launch(gamer_hydro_t h, const gamer_hierarchy_t* H) {
    DiagArgs<T> a;
    diag_args<T>(h, H, a);
    CK(h, launch_diag<T>(a, h->total_groups, h->stream));
    return GAMER_OK;
}

int diagnose_impl(gamer_hydro_t h, const gamer_hierarchy_t* H, double cfl, double* dt_out,
                  double* sums, int64_t* n_bad) {
    int r = prepare(h, H);
    if (r) return r;
    if ((r = check_pointers(h, H, false))) return r;
    r = h->precision == GAMER_FP32 ? diag_launch<float>(h, H) : diag_launch<double>(h, H);
    if (r) return r;
    CK(h, cudaMemcpyAsync(h->h_out, h->d_out, sizeof(DiagOut) * H->n_levels, cudaMemcpyDeviceToHost,
                          h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (dt_out) {
        double dt = INFINITY;
        for (int l = 0; l < H->n_levels; ++l) {
            if (H->levels[l].n_groups == 0) continue;
            unsigned long long b = h->h_out[l].smax_bits;
            double s;
            memcpy(&s, &b, sizeof(s));
            // individual time steps: level l takes 2^l steps per dt
            double d = (h->individual ? std::ldexp(H->levels[l].dh, l) : H->levels[l].dh) / s;
            if (d < dt || d != d) dt = d;
        }
        *dt_out = cfl * dt;
    }
    if (sums) {
        for (int v = 0; v < NV; ++v) sums[v] = 0.0;
        for (int l = 0; l < H->n_levels; ++l) {
            const double dh = H->levels[l].dh, dV = dh * dh * dh;
            for (int v = 0; v < NV; ++v) sums[v] += h->h_out[l].sum[v] * dV;
        }
    }
    if (n_bad) {
        long long nb = 0;
        for (int l = 0; l < H->n_levels; ++l) nb += h->h_out[l].n_bad;
        *n_bad = nb;
    }
    return GAMER_OK;
}

int check_same_parity(gamer_hydro_t h, const gamer_hierarchy_t* H) {
    for (int l = 1; l < H->n_levels; ++l)
        if (h->parity[l] != h->parity[0])
            return fail(h, GAMER_ERR_STATE, "a whole step needs every level at the same sweep parity");
    return GAMER_OK;
}

// Launch sequence of one whole step on stream st (dt read from h->d_dt):
// every level's sweep set (the FP32 handle: one persistent launch over the
// groups of all levels), the fix-ups from the finest level down, and, when
// `with_diag`, the diagnostics of the new state and the step result (new
// dt from Eq. CFL, held if the next step is a zyx step) with its copy to
// pinned host memory.  Single-level FP32 steps fuse the per-group
// diagnostics into the sweep launch.
int enqueue_step(gamer_hydro_t h, const gamer_hierarchy_t* H, cudaStream_t st, bool with_diag, double cfl) {
    const int n = H->n_levels;
    const int order = h->parity[0];
    cudaStream_t saved = h->stream;
    h->stream = st;
    int r = GAMER_OK;
    const bool fused = with_diag && h->precision == GAMER_FP32 && n == 1;
    bool reduced = false;   // the sweep launch runs the end-of-step reduction itself
    DiagArgs<float> d32;
    DiagArgs<double> d64;
    if (h->precision == GAMER_FP32) {
        SweepArgs<float> a;
        memset(&a, 0, sizeof(a));
        int item = 0;
        for (int l = 0; l < n; ++l) {
            fill_level<float>(a.lv[l], H->levels, l, h);
            a.lv[l].item0 = item;
            item += H->levels[l].n_groups;
        }
        a.n_levels = n;
        a.total = item;
        a.queue = h->d_queue;
        a.done = reinterpret_cast<unsigned*>(h->d_queue + 1);
        a.dt = h->d_dt;
        a.gamma = (float)h->gamma;
        a.gm1 = (float)(h->gamma - 1.0);
        if (fused) a.diag = DiagSink{h->d_pg_max, h->d_pg_sum, h->d_pg_bad};
        // the next step is an xyz step exactly when this one is zyx
        reduced = fused && item > 0;
        if (reduced)
            a.step = StepSink{h->d_step, h->h_step_dev, h->d_dt, cfl, H->levels[0].dh, order == 1, item};
        if (item > 0) {
            cudaError_t e = cudaSuccess;
            if (h->prof_ev[0]) e = cudaEventRecord(h->prof_ev[0], st);
            if (e == cudaSuccess)
                e = launch_sweep_f32(a, order, h->limiter, h->f32_variant, h->sweep_threads, sweep_grid(h, item), st);
            if (e == cudaSuccess && h->prof_ev[1]) e = cudaEventRecord(h->prof_ev[1], st);
            if (e != cudaSuccess) r = cuda_fail(h, e, "FP32 sweep launch");
        }
    } else {
        if (h->prof_ev[0]) {
            cudaError_t e = cudaEventRecord(h->prof_ev[0], st);
            if (e != cudaSuccess) r = cuda_fail(h, e, "cudaEventRecord");
        }
        for (int l = 0; l < n && !r; ++l) r = advance_level_impl(h, H, l, order);
        if (!r && h->prof_ev[1]) {
            cudaError_t e = cudaEventRecord(h->prof_ev[1], st);
            if (e != cudaSuccess) r = cuda_fail(h, e, "cudaEventRecord");
        }
    }
    for (int l = n - 2; l >= 0 && !r; --l) r = fixup_impl(h, H, l);
    if (!r && with_diag) {
        // the diagnostics read the new state: u_out of every level
        gamer_level_t lv[MAXLEV];
        for (int l = 0; l < n; ++l) {
            lv[l] = H->levels[l];
            lv[l].u = H->levels[l].u_out;
        }
        gamer_hierarchy_t Hn = *H;
        Hn.levels = lv;
        double dh[MAXLEV];
        for (int l = 0; l < n; ++l) dh[l] = H->levels[l].dh;
        diag_args<float>(h, &Hn, d32);
        diag_args<double>(h, &Hn, d64);
        cudaError_t e = cudaSuccess;
        if (!fused)
            e = h->precision == GAMER_FP32 ? launch_diag_groups<float>(d32, h->total_groups, st)
                                           : launch_diag_groups<double>(d64, h->total_groups, st);
        if (e == cudaSuccess && !reduced)
            e = launch_step_final(d32, d64, h->precision == GAMER_FP64, dh, nullptr, cfl, h->d_dt, order == 1,
                                  h->d_step, h->h_step_dev, st);
        if (e != cudaSuccess) r = cuda_fail(h, e, "step diagnostics");
    }
    h->stream = saved;
    return r;
}

// Individual time steps (Sec. 2.1; readings R18-R20): two steps of level l
// with dt0 / 2^l, each its sweep set (u -> u_out; coarse ghosts
// interpolated in time, weight 0 then 1/2), then the two steps of the finer
// level, then this level's fix-up from it, then u <-> u_out in lv.  Level
// l's fluxes go to its own buffer in its first step and to the second
// buffer in its second step; the fix-up averages the finer level's two.
int cycle_level(gamer_hydro_t h, gamer_level_t* lv, const gamer_hierarchy_t* Hc, int l) {
    const int n = Hc->n_levels;
    auto flux_of = [&](int lev, int k) -> void* {
        if (k == 1) return h->lv[lev].own_flux2;
        return lv[lev].face_flux ? lv[lev].face_flux : h->lv[lev].own_flux;
    };
    for (int k = 0; k < 2; ++k) {
        LevelStep ls;
        ls.dts = std::ldexp(1.0, -l);
        ls.cw = (l > 0 && k == 1) ? 0.5 : 0.0;
        ls.ucn = (l > 0 && k == 1) ? lv[l - 1].u_out : nullptr;
        ls.flux = flux_of(l, k);
        int r = advance_level_impl(h, Hc, l, k, &ls);
        if (r) return r;
        if (l + 1 < n) {
            if ((r = cycle_level(h, lv, Hc, l + 1))) return r;
            FixStep fs;
            fs.fc = flux_of(l, k);
            fs.ff = flux_of(l + 1, 0);
            fs.ff2 = flux_of(l + 1, 1);
            fs.uf = lv[l + 1].u;          // the finer state after its two steps
            fs.dts = std::ldexp(1.0, -l);
            if ((r = fixup_impl(h, Hc, l, &fs))) return r;
        }
        void* t = lv[l].u_out;
        lv[l].u_out = const_cast<void*>(lv[l].u);
        lv[l].u = t;
    }
    return GAMER_OK;
}

// Launch sequence of one individual-time-step cycle of a multi-level
// hierarchy on stream st (two level-0 steps with one dt), every level back
// in u, then the diagnostics and the next dt (Eq. CFL with the 2^l factors).
int enqueue_cycle(gamer_hydro_t h, const gamer_hierarchy_t* H, cudaStream_t st, double cfl) {
    cudaStream_t saved = h->stream;
    h->stream = st;
    gamer_level_t lv[MAXLEV];
    for (int l = 0; l < H->n_levels; ++l) lv[l] = H->levels[l];
    gamer_hierarchy_t Hc = *H;
    Hc.levels = lv;
    int r = GAMER_OK;
    cudaError_t e = cudaSuccess;
    if (h->prof_ev[0]) e = cudaEventRecord(h->prof_ev[0], st);
    if (e != cudaSuccess) r = cuda_fail(h, e, "cudaEventRecord");
    if (!r) r = cycle_level(h, lv, &Hc, 0);
    if (!r && h->prof_ev[1]) {
        e = cudaEventRecord(h->prof_ev[1], st);
        if (e != cudaSuccess) r = cuda_fail(h, e, "cudaEventRecord");
    }
    if (!r) {
        DiagArgs<float> d32;
        DiagArgs<double> d64;
        diag_args<float>(h, H, d32);      // every level's new state is in u
        diag_args<double>(h, H, d64);
        double dh[MAXLEV], ds[MAXLEV];
        for (int l = 0; l < H->n_levels; ++l) {
            dh[l] = H->levels[l].dh;
            ds[l] = std::ldexp(1.0, l);
        }
        e = h->precision == GAMER_FP32 ? launch_diag_groups<float>(d32, h->total_groups, st)
                                       : launch_diag_groups<double>(d64, h->total_groups, st);
        if (e == cudaSuccess)
            e = launch_step_final(d32, d64, h->precision == GAMER_FP64, dh, ds, cfl, h->d_dt, 1, h->d_step,
                                  h->h_step_dev, st);
        if (e != cudaSuccess) r = cuda_fail(h, e, "cycle diagnostics");
    }
    h->stream = saved;
    return r;
}

// The hierarchy with u and u_out exchanged on every level (the second set
// of a pair when it runs as two steps).
struct SwappedHierarchy {
    gamer_level_t lv[MAXLEV];
    gamer_hierarchy_t H;
    explicit SwappedHierarchy(const gamer_hierarchy_t* src) {
        for (int l = 0; l < src->n_levels; ++l) {
            lv[l] = src->levels[l];
            lv[l].u = src->levels[l].u_out;
            lv[l].u_out = const_cast<void*>(src->levels[l].u);
        }
        H = *src;
        H.levels = lv;
    }
};

// Launch sequence of one sweep-set pair (xyz then zyx, same dt) on stream
// st, the result back in u.  One level in FP32: a single pair launch whose
// last CTA also reduces the diagnostics and writes dt and the step result.
// Otherwise: two whole steps, the second on the swapped hierarchy.
int enqueue_pair(gamer_hydro_t h, const gamer_hierarchy_t* H, cudaStream_t st, double cfl) {
    if (h->individual && H->n_levels > 1) return enqueue_cycle(h, H, st, cfl);
    const int n = H->levels[0].n_groups;
    if (!(h->precision == GAMER_FP32 && H->n_levels == 1 && n > 0 && h->pair_n == n)) {
        // the xyz set keeps dt and its state is not the pair's result: no
        // diagnostics after it, as in the fused pair launch
        int r = enqueue_step(h, H, st, false, cfl);
        if (r) return r;
        for (int l = 0; l < H->n_levels; ++l) h->parity[l] ^= 1;
        SwappedHierarchy S(H);
        r = enqueue_step(h, &S.H, st, true, cfl);
        for (int l = 0; l < H->n_levels; ++l) h->parity[l] ^= 1;
        return r;
    }
    SweepArgs<float> a;
    memset(&a, 0, sizeof(a));
    fill_level<float>(a.lv[0], H->levels, 0, h);
    SwappedHierarchy S(H);
    fill_level<float>(a.lv[1], S.H.levels, 0, h);
    a.lv[0].item0 = 0;
    a.lv[1].item0 = n;
    a.n_levels = 2;
    a.total = 2 * n;
    a.queue = h->d_queue;
    a.done = reinterpret_cast<unsigned*>(h->d_queue + 1);
    a.dt = h->d_dt;
    a.gamma = (float)h->gamma;
    a.gm1 = (float)(h->gamma - 1.0);
    a.diag = DiagSink{h->d_pg_max, h->d_pg_sum, h->d_pg_bad};
    // after a zyx set the next set is an xyz set: take the new dt
    a.step = StepSink{h->d_step, h->h_step_dev, h->d_dt, cfl, H->levels[0].dh, 1, n};
    a.pair = PairArgs{h->d_ready, reinterpret_cast<unsigned*>(h->d_queue + 2),
                      reinterpret_cast<unsigned*>(h->d_queue + 3), h->d_order1, h->hold};
    cudaError_t e = cudaSuccess;
    if (h->prof_ev[0]) e = cudaEventRecord(h->prof_ev[0], st);
    if (e == cudaSuccess) e = launch_sweep_pair(a, h->limiter, std::max(1, std::min(2 * n, h->sm_count)), st);
    if (e == cudaSuccess && h->prof_ev[1]) e = cudaEventRecord(h->prof_ev[1], st);
    if (e != cudaSuccess) return cuda_fail(h, e, "FP32 pair launch");
    return GAMER_OK;
}

// dt of the current state (Eq. CFL) into h->d_dt, on the handle's stream.
int diagnose_to_device(gamer_hydro_t h, const gamer_hierarchy_t* H, double cfl) {
    DiagArgs<float> d32;
    DiagArgs<double> d64;
    diag_args<float>(h, H, d32);
    diag_args<double>(h, H, d64);
    double dh[MAXLEV], ds[MAXLEV];
    for (int l = 0; l < H->n_levels; ++l) {
        dh[l] = H->levels[l].dh;
        ds[l] = std::ldexp(1.0, l);
    }
    cudaError_t e = h->precision == GAMER_FP32 ? launch_diag_groups<float>(d32, h->total_groups, h->stream)
                                               : launch_diag_groups<double>(d64, h->total_groups, h->stream);
    if (e == cudaSuccess)
        e = launch_step_final(d32, d64, h->precision == GAMER_FP64, dh, h->individual ? ds : nullptr, cfl,
                              h->d_dt, 1, h->d_step, nullptr, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "initial CFL time step");
    return GAMER_OK;
}

}  // namespace

// =================================================================== C ABI

extern "C" {

int gamer_hydro_create(double gamma, int limiter, int ghost_width, int precision, gamer_hydro_t* out) {
    if (!out) return fail(nullptr, GAMER_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!(gamma > 1.0) || !std::isfinite(gamma)) return fail(nullptr, GAMER_ERR_ARG, "gamma must be > 1");
    if (limiter != GAMER_LIMITER_VANLEER && limiter != GAMER_LIMITER_MINMOD)
        return fail(nullptr, GAMER_ERR_ARG, "unknown limiter");
    if (precision != GAMER_FP32 && precision != GAMER_FP64)
        return fail(nullptr, GAMER_ERR_ARG, "unknown precision");
    if (ghost_width != NG)
        return fail(nullptr, GAMER_ERR_UNSUPPORTED, "ghost_width must be 3 (seven-point stencil)");
    gamer_hydro_t h = new gamer_hydro_s();
    h->gamma = gamma;
    h->limiter = limiter;
    h->precision = precision;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
    // work-queue counter and finished-CTA counter: zeroed once here, set back
    // to zero by the last CTA of every FP32 sweep launch; then the pair
    // launch counter and the pair wait-status word
    if (e == cudaSuccess) e = cudaMalloc(&h->d_queue, 4 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->d_queue, 0, 4 * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_dt, sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_step, sizeof(StepOut));
    if (e == cudaSuccess) e = cudaMemset(h->d_step, 0, sizeof(StepOut));
    if (e == cudaSuccess) e = cudaHostAlloc(&h->h_step, sizeof(StepOut), cudaHostAllocMapped);
    if (e == cudaSuccess) memset(h->h_step, 0, sizeof(StepOut));
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(&h->h_step_dev, h->h_step, 0);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->step_event, cudaEventDisableTiming);
    if (e == cudaSuccess) e = sweep_f32_init();
    if (e != cudaSuccess) {
        std::string m = std::string("CUDA initialisation failed: ") + cudaGetErrorString(e);
        cudaFree(h->d_queue);
        cudaFree(h->d_dt);
        cudaFree(h->d_step);
        cudaFreeHost(h->h_step);
        if (h->step_event) cudaEventDestroy(h->step_event);
        delete h;
        return fail(nullptr, GAMER_ERR_CUDA, m);
    }
    *out = h;
    return GAMER_OK;
}

int gamer_hydro_destroy(gamer_hydro_t h) {
    if (!h) return GAMER_OK;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    drop_hierarchy(h);
    cudaFree(h->d_queue);
    cudaFree(h->d_ready);
    cudaFree(h->d_order1);
    cudaFree(h->d_dt);
    cudaFree(h->d_pg_max);
    cudaFree(h->d_pg_sum);
    cudaFree(h->d_pg_bad);
    cudaFree(h->d_out);
    cudaFreeHost(h->h_out);
    cudaFree(h->d_stage);
    cudaFree(h->d_step);
    cudaFreeHost(h->h_step);
    if (h->step_event) cudaEventDestroy(h->step_event);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    delete h;
    return GAMER_OK;
}

int gamer_hydro_set_stream(gamer_hydro_t h, void* s) {
    if (!h) return GAMER_ERR_ARG;
    h->stream = static_cast<cudaStream_t>(s);
    drop_graphs(h);
    return GAMER_OK;
}

int gamer_hydro_set_parity(gamer_hydro_t h, int level, int parity) {
    if (!h) return GAMER_ERR_ARG;
    if (level < 0 || level >= 32 || (parity != 0 && parity != 1))
        return fail(h, GAMER_ERR_ARG, "level must be in [0,32) and parity 0 or 1");
    h->parity[level] = parity;
    return GAMER_OK;
}

int gamer_poisson_prepare(gamer_hydro_t h, const gamer_hierarchy_t* H, int level, const void* phi_c,
                          void* phi_blocks, void* rho_blocks) {
    if (!h) return GAMER_ERR_ARG;
    if (!phi_c || !phi_blocks || !rho_blocks)
        return fail(h, GAMER_ERR_ARG, "phi_c, phi_blocks and rho_blocks are required");
    CK(h, cudaSetDevice(h->device));
    int r = prepare(h, H);
    if (r) return r;
    if ((r = check_level_arg(h, H, level))) return r;
    if (level < 1) return fail(h, GAMER_ERR_ARG, "level 0 has no coarser level to take the boundary from");
    const gamer_level_t& L = H->levels[level];
    const gamer_level_t& C = H->levels[level - 1];
    if (L.n_groups == 0) return GAMER_OK;
    if (!L.u) return fail(h, GAMER_ERR_ARG, "u is NULL");
    if (h->precision == GAMER_FP32) {
        PrepArgs<float> a{static_cast<const float*>(phi_c), C.nbr, C.n_groups, L.parent,
                          static_cast<const float*>(L.u), L.n_groups, static_cast<float*>(phi_blocks),
                          static_cast<float*>(rho_blocks)};
        CK(h, launch_poisson_prepare<float>(a, h->stream));
    } else {
        PrepArgs<double> a{static_cast<const double*>(phi_c), C.nbr, C.n_groups, L.parent,
                           static_cast<const double*>(L.u), L.n_groups, static_cast<double*>(phi_blocks),
                           static_cast<double*>(rho_blocks)};
        CK(h, launch_poisson_prepare<double>(a, h->stream));
    }
    return GAMER_OK;
}

int gamer_hydro_test_withhold(gamer_hydro_t h, int group) {
    if (!h) return GAMER_ERR_ARG;
    if (group < -1) return fail(h, GAMER_ERR_ARG, "group must be -1 or a patch group of level 0");
    h->hold = group;
    return GAMER_OK;
}

int gamer_hydro_set_launch_groups(gamer_hydro_t h, int n) {
    if (!h) return GAMER_ERR_ARG;
    if (n < 1) return fail(h, GAMER_ERR_ARG, "groups per launch must be >= 1");
    if (h->precision != GAMER_FP64) return fail(h, GAMER_ERR_UNSUPPORTED, "groups per launch applies to FP64 handles");
    if (n != h->f64_chunk) {
        CK(h, cudaSetDevice(h->device));
        if (h->stream) CK(h, cudaStreamSynchronize(h->stream));
        else CK(h, cudaDeviceSynchronize());
        h->f64_chunk = n;
        drop_hierarchy(h);            // captured graphs hold the old launch sequence
    }
    return GAMER_OK;
}

int gamer_hydro_set_time_steps(gamer_hydro_t h, int mode) {
    if (!h) return GAMER_ERR_ARG;
    if (mode != GAMER_TIME_STEPS_UNIFORM && mode != GAMER_TIME_STEPS_INDIVIDUAL)
        return fail(h, GAMER_ERR_ARG, "unknown time-step mode");
    if (mode != h->individual) {
        CK(h, cudaSetDevice(h->device));
        if (h->stream) CK(h, cudaStreamSynchronize(h->stream));
        else CK(h, cudaDeviceSynchronize());
        h->individual = mode;
        drop_hierarchy(h);            // buffers and graphs depend on the mode
        h->dt_ready = false;          // and so does Eq. CFL
    }
    return GAMER_OK;
}

int gamer_hydro_flag(gamer_hydro_t h, const gamer_hierarchy_t* H, int level, int criterion, double threshold,
                     int n_buffer, uint32_t* masks) {
    if (!h) return GAMER_ERR_ARG;
    if (criterion < GAMER_FLAG_DENSITY_GRADIENT || criterion > GAMER_FLAG_DENSITY)
        return fail(h, GAMER_ERR_ARG, "unknown refinement criterion");
    if (n_buffer < 0 || n_buffer > PS) return fail(h, GAMER_ERR_ARG, "n_buffer must be in [0, 8]");
    if (!masks) return fail(h, GAMER_ERR_ARG, "masks is NULL");
    CK(h, cudaSetDevice(h->device));
    int r = prepare(h, H);
    if (r) return r;
    if ((r = check_level_arg(h, H, level))) return r;
    const gamer_level_t& L = H->levels[level];
    if (L.n_groups == 0) return GAMER_OK;
    if (!L.u) return fail(h, GAMER_ERR_ARG, "u is NULL");
    if (h->precision == GAMER_FP32) {
        FlagArgs<float> a{static_cast<const float*>(L.u), L.nbr, L.n_groups, criterion, threshold, n_buffer,
                          h->gamma, masks};
        CK(h, launch_flag<float>(a, h->stream));
    } else {
        FlagArgs<double> a{static_cast<const double*>(L.u), L.nbr, L.n_groups, criterion, threshold, n_buffer,
                           h->gamma, masks};
        CK(h, launch_flag<double>(a, h->stream));
    }
    return GAMER_OK;
}

int gamer_hydro_refine_fill(gamer_hydro_t h, const gamer_hierarchy_t* H, int level, int n_new,
                            const int32_t* parent_new, const int32_t* inherit, const void* u_old, int n_old,
                            void* u_new) {
    if (!h) return GAMER_ERR_ARG;
    if (n_new < 0 || n_old < 0) return fail(h, GAMER_ERR_ARG, "negative group count");
    if (n_new == 0) return GAMER_OK;
    if (!parent_new || !inherit || !u_new) return fail(h, GAMER_ERR_ARG, "parent_new, inherit and u_new are required");
    if (reinterpret_cast<uintptr_t>(u_new) % 16 || reinterpret_cast<uintptr_t>(u_old) % 16)
        return fail(h, GAMER_ERR_ARG, "u_new and u_old must be 16-byte aligned");
    CK(h, cudaSetDevice(h->device));
    int r = prepare(h, H);
    if (r) return r;
    if ((r = check_level_arg(h, H, level))) return r;
    const gamer_level_t& L = H->levels[level];
    if (!L.u) return fail(h, GAMER_ERR_ARG, "u is NULL");
    // validate on the host: parents in range and properly nested (the 26
    // neighbours of every parent patch exist on its level), inheritance in range
    std::vector<int> par(n_new), inh(n_new), nbr((size_t)L.n_groups * 26);
    CK(h, cudaMemcpy(par.data(), parent_new, sizeof(int) * n_new, cudaMemcpyDeviceToHost));
    CK(h, cudaMemcpy(inh.data(), inherit, sizeof(int) * n_new, cudaMemcpyDeviceToHost));
    CK(h, cudaMemcpy(nbr.data(), L.nbr, sizeof(int) * nbr.size(), cudaMemcpyDeviceToHost));
    for (int i = 0; i < n_new; ++i) {
        if (inh[i] >= n_old || inh[i] < -1) return fail(h, GAMER_ERR_ARG, "inherit entry out of range");
        if (inh[i] >= 0) {
            if (!u_old) return fail(h, GAMER_ERR_ARG, "u_old is NULL but groups inherit");
            continue;
        }
        const int P = par[i];
        if (P < 0 || P >= 8 * L.n_groups) return fail(h, GAMER_ERR_MAP, "parent_new entry out of range");
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int lp = P & 7;
                    int q[3] = {(lp & 1) + dx, ((lp >> 1) & 1) + dy, ((lp >> 2) & 1) + dz};
                    if (resolve_patch(nbr, P >> 3, q) < 0)
                        return fail(h, GAMER_ERR_MAP, "a parent patch of the new level is not properly nested");
                }
    }
    if (h->precision == GAMER_FP32) {
        RefineArgs<float> a{static_cast<const float*>(L.u), L.nbr, L.n_groups, parent_new, inherit,
                            static_cast<const float*>(u_old), n_old, static_cast<float*>(u_new), n_new};
        CK(h, launch_refine<float>(a, h->stream));
    } else {
        RefineArgs<double> a{static_cast<const double*>(L.u), L.nbr, L.n_groups, parent_new, inherit,
                             static_cast<const double*>(u_old), n_old, static_cast<double*>(u_new), n_new};
        CK(h, launch_refine<double>(a, h->stream));
    }
    return GAMER_OK;
}

int gamer_hydro_get_parity(gamer_hydro_t h, int level, int* parity) {
    if (!h || !parity) return GAMER_ERR_ARG;
    if (level < 0 || level >= 32) return fail(h, GAMER_ERR_ARG, "level must be in [0,32)");
    *parity = h->parity[level];
    return GAMER_OK;
}

int gamer_hydro_cfl_dt(gamer_hydro_t h, const gamer_hierarchy_t* H, double cfl, double* dt_out) {
    if (!h) return GAMER_ERR_ARG;
    if (!dt_out) return fail(h, GAMER_ERR_ARG, "dt_out is NULL");
    if (!(cfl > 0.0)) return fail(h, GAMER_ERR_ARG, "cfl must be positive");
    CK(h, cudaSetDevice(h->device));
    return diagnose_impl(h, H, cfl, dt_out, nullptr, nullptr);
}

int gamer_hydro_check(gamer_hydro_t h, const gamer_hierarchy_t* H, double sums[5], int64_t* n_bad) {
    if (!h) return GAMER_ERR_ARG;
    if (!sums || !n_bad) return fail(h, GAMER_ERR_ARG, "sums and n_bad are required");
    CK(h, cudaSetDevice(h->device));
    return diagnose_impl(h, H, 1.0, nullptr, sums, n_bad);
}

int gamer_hydro_diagnose(gamer_hydro_t h, const gamer_hierarchy_t* H, double cfl, double* dt_out,
                         double sums[5], int64_t* n_bad) {
    if (!h) return GAMER_ERR_ARG;
    if (dt_out && !(cfl > 0.0)) return fail(h, GAMER_ERR_ARG, "cfl must be positive");
    CK(h, cudaSetDevice(h->device));
    return diagnose_impl(h, H, cfl, dt_out, sums, n_bad);
}

int gamer_hydro_advance(gamer_hydro_t h, const gamer_hierarchy_t* H, int level, double dt) {
    if (!h) return GAMER_ERR_ARG;
    if (!(dt >= 0.0) || !std::isfinite(dt)) return fail(h, GAMER_ERR_ARG, "dt must be finite and >= 0");
    CK(h, cudaSetDevice(h->device));
    int r = prepare(h, H);
    if (r) return r;
    if ((r = check_level_arg(h, H, level))) return r;
    if ((r = check_pointers(h, H, true))) return r;
    CK(h, launch_set_dt(h->d_dt, dt, h->stream));
    h->dt_ready = false;
    r = advance_level_impl(h, H, level, h->parity[level]);
    if (r) return r;
    h->parity[level] ^= 1;
    return GAMER_OK;
}

int gamer_hydro_fixup(gamer_hydro_t h, const gamer_hierarchy_t* H, int level, double dt) {
    if (!h) return GAMER_ERR_ARG;
    if (!(dt >= 0.0) || !std::isfinite(dt)) return fail(h, GAMER_ERR_ARG, "dt must be finite and >= 0");
    CK(h, cudaSetDevice(h->device));
    int r = prepare(h, H);
    if (r) return r;
    if ((r = check_pointers(h, H, true))) return r;
    if (level < 0 || level + 1 >= H->n_levels)
        return fail(h, GAMER_ERR_ARG, "fixup level must be in [0, n_levels-2]");
    CK(h, launch_set_dt(h->d_dt, dt, h->stream));
    h->dt_ready = false;
    return fixup_impl(h, H, level);
}

int gamer_hydro_advance_all(gamer_hydro_t h, const gamer_hierarchy_t* H, double dt) {
    if (!h) return GAMER_ERR_ARG;
    if (!(dt >= 0.0) || !std::isfinite(dt)) return fail(h, GAMER_ERR_ARG, "dt must be finite and >= 0");
    CK(h, cudaSetDevice(h->device));
    int r = prepare(h, H);
    if (r) return r;
    if ((r = check_pointers(h, H, true))) return r;
    if ((r = check_same_parity(h, H))) return r;
    CK(h, launch_set_dt(h->d_dt, dt, h->stream));
    h->dt_ready = false;
    if ((r = enqueue_step(h, H, h->stream, false, 0.0))) return r;
    for (int l = 0; l < H->n_levels; ++l) h->parity[l] ^= 1;
    return GAMER_OK;
}

int gamer_hydro_step(gamer_hydro_t h, const gamer_hierarchy_t* H, double cfl) {
    if (!h) return GAMER_ERR_ARG;
    if (!(cfl > 0.0) || !std::isfinite(cfl)) return fail(h, GAMER_ERR_ARG, "cfl must be positive");
    if (H && h->individual && H->n_levels > 1)
        return fail(h, GAMER_ERR_UNSUPPORTED, "individual time steps advance in pairs: use gamer_hydro_step_pair");
    CK(h, cudaSetDevice(h->device));
    int r = prepare(h, H);
    if (r) return r;
    if ((r = check_pointers(h, H, true))) return r;
    if ((r = check_same_parity(h, H))) return r;
    if (!h->dt_ready || h->dt_version != h->version) {
        // first step on this state: dt from Eq. CFL of the current state
        if ((r = diagnose_to_device(h, H, cfl))) return r;
        h->dt_ready = true;
        h->dt_version = h->version;
    }
    if (h->prof_ev[0]) {
        // profiled steps launch directly: events recorded inside a graph
        // cannot be timed
        if ((r = enqueue_step(h, H, h->stream, true, cfl))) return r;
        CK(h, cudaEventRecord(h->step_event, h->stream));
        for (int l = 0; l < H->n_levels; ++l) h->parity[l] ^= 1;
        return GAMER_OK;
    }
    // graph of the whole step, keyed by everything the kernels are given
    char key[64];
    std::string k;
    snprintf(key, sizeof(key), "%llu|%d|%.17g|", (unsigned long long)h->version, h->parity[0], cfl);
    k = key;
    for (int l = 0; l < H->n_levels; ++l) {
        snprintf(key, sizeof(key), "%p,%p,%p;", H->levels[l].u, H->levels[l].u_out, H->levels[l].face_flux);
        k += key;
    }
    auto it = h->graphs.find(k);
    if (it == h->graphs.end()) {
        if (!h->cap_stream) CK(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
        if (h->graphs.size() >= 16) drop_graphs(h);
        cudaGraph_t graph = nullptr;
        CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
        r = enqueue_step(h, H, h->cap_stream, true, cfl);
        cudaError_t e = cudaStreamEndCapture(h->cap_stream, &graph);
        if (r) {
            if (graph) cudaGraphDestroy(graph);
            return r;
        }
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
        GraphEntry ge;
        e = cudaGraphInstantiate(&ge.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
        it = h->graphs.emplace(k, ge).first;
    }
    it->second.last_use = ++h->use_clock;
    CK(h, cudaGraphLaunch(it->second.exec, h->stream));
    CK(h, cudaEventRecord(h->step_event, h->stream));
    for (int l = 0; l < H->n_levels; ++l) h->parity[l] ^= 1;
    return GAMER_OK;
}

int gamer_hydro_step_pair(gamer_hydro_t h, const gamer_hierarchy_t* H, double cfl) {
    if (!h) return GAMER_ERR_ARG;
    if (!(cfl > 0.0) || !std::isfinite(cfl)) return fail(h, GAMER_ERR_ARG, "cfl must be positive");
    CK(h, cudaSetDevice(h->device));
    int r = prepare(h, H);
    if (r) return r;
    if ((r = check_pointers(h, H, true))) return r;
    if ((r = check_same_parity(h, H))) return r;
    if (h->parity[0] != 0) return fail(h, GAMER_ERR_STATE, "a sweep-set pair starts with an xyz set (parity 0)");
    if (!h->dt_ready || h->dt_version != h->version) {
        if ((r = diagnose_to_device(h, H, cfl))) return r;
        h->dt_ready = true;
        h->dt_version = h->version;
    }
    if (h->prof_ev[0] || h->hold >= 0) {
        // launched directly: profiling events cannot be timed inside graphs,
        // and a withheld mark is a one-off that no graph should keep
        r = enqueue_pair(h, H, h->stream, cfl);
        h->hold = -1;
        if (r) return r;
        CK(h, cudaEventRecord(h->step_event, h->stream));
        return GAMER_OK;
    }
    char key[64];
    snprintf(key, sizeof(key), "pair%d|%llu|%.17g|", h->individual, (unsigned long long)h->version, cfl);
    std::string k = key;
    for (int l = 0; l < H->n_levels; ++l) {
        snprintf(key, sizeof(key), "%p,%p,%p;", H->levels[l].u, H->levels[l].u_out, H->levels[l].face_flux);
        k += key;
    }
    auto it = h->graphs.find(k);
    if (it == h->graphs.end()) {
        if (!h->cap_stream) CK(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
        if (h->graphs.size() >= 16) drop_graphs(h);
        cudaGraph_t graph = nullptr;
        CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
        r = enqueue_pair(h, H, h->cap_stream, cfl);
        cudaError_t e = cudaStreamEndCapture(h->cap_stream, &graph);
        if (r) {
            if (graph) cudaGraphDestroy(graph);
            return r;
        }
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
        GraphEntry ge;
        e = cudaGraphInstantiate(&ge.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
        it = h->graphs.emplace(k, ge).first;
    }
    it->second.last_use = ++h->use_clock;
    CK(h, cudaGraphLaunch(it->second.exec, h->stream));
    CK(h, cudaEventRecord(h->step_event, h->stream));
    return GAMER_OK;
}

int gamer_hydro_step_result(gamer_hydro_t h, double* dt_used, double* dt_next, double sums[5],
                            int64_t* n_bad) {
    if (!h) return GAMER_ERR_ARG;
    CK(h, cudaSetDevice(h->device));
    CK(h, cudaEventSynchronize(h->step_event));
    const StepOut& o = *h->h_step;
    if (o.steps == 0) return fail(h, GAMER_ERR_STATE, "no step has completed on this handle");
    if (o.status != 0) {
        h->dt_ready = false;          // the dt that launch left is not trusted: the next step takes Eq. CFL anew
        return fail(h, GAMER_ERR_TIMEOUT, "a dependency wait of the last pair launch gave up; its result is invalid");
    }
    if (dt_used) *dt_used = o.dt_used;
    if (dt_next) *dt_next = o.dt_next;
    if (sums)
        for (int v = 0; v < NV; ++v) sums[v] = o.sum[v];
    if (n_bad) *n_bad = o.n_bad;
    return GAMER_OK;
}

int gamer_hydro_tune(gamer_hydro_t h, const gamer_hierarchy_t* H, const char* cache_path) {
    if (!h) return GAMER_ERR_ARG;
    CK(h, cudaSetDevice(h->device));
    int r = prepare(h, H);
    if (r) return r;
    if ((r = check_pointers(h, H, true))) return r;
    if ((r = check_same_parity(h, H))) return r;
    cudaDeviceProp prop;
    CK(h, cudaGetDeviceProperties(&prop, h->device));
    int bucket = 0;
    while ((1 << bucket) < h->total_groups) ++bucket;
    char key[384];
    snprintf(key, sizeof(key), "%s|%s|lim%d|levels%d|groups2^%d", prop.name,
             h->precision == GAMER_FP32 ? "fp32" : "fp64", h->limiter, H->n_levels, bucket);
    for (char* c = key; *c; ++c)
        if (*c == ' ' || *c == '=') *c = '_';
    struct Cand { int variant, threads, grid, f64t; };
    std::vector<Cand> cands;
    if (h->precision == GAMER_FP32)
        cands = {{0, 512, 0, 256}, {0, 512, 1, 256}, {1, 512, 0, 256}, {1, 256, 0, 256}, {1, 512, 1, 256}};
    else
        cands = {{0, 512, 0, 256}, {0, 512, 0, 128}};
    auto apply = [&](const Cand& c) {
        h->f32_variant = c.variant;
        h->sweep_threads = c.threads;
        h->grid_mode = c.grid;
        h->f64_threads = c.f64t;
    };
    if (cache_path) {
        FILE* f = fopen(cache_path, "r");
        if (f) {
            char line[512];
            while (fgets(line, sizeof(line), f)) {
                char* eq = strrchr(line, '=');
                if (!eq) continue;
                *eq = 0;
                Cand c;
                if (strcmp(line, key) == 0 && sscanf(eq + 1, "%d,%d,%d,%d", &c.variant, &c.threads, &c.grid, &c.f64t) == 4) {
                    bool known = false;
                    for (const Cand& k : cands)
                        known |= k.variant == c.variant && k.threads == c.threads && k.grid == c.grid && k.f64t == c.f64t;
                    if (known) {
                        fclose(f);
                        apply(c);
                        h->tuned = true;
                        drop_graphs(h);
                        return GAMER_OK;
                    }
                }
            }
            fclose(f);
        }
    }
    // time every candidate on this hierarchy: dt = 0 keeps the arithmetic
    // and overwrites u_out (and face fluxes), never u
    CK(h, launch_set_dt(h->d_dt, 0.0, h->stream));
    h->dt_ready = false;
    cudaEvent_t e0, e1;
    CK(h, cudaEventCreate(&e0));
    CK(h, cudaEventCreate(&e1));
    float best = 1e30f;
    Cand pick = cands[0];
    for (const Cand& c : cands) {
        apply(c);
        float t = 1e30f;
        for (int rep = 0; rep < 4 && !r; ++rep) {
            cudaEventRecord(e0, h->stream);
            r = enqueue_step(h, H, h->stream, false, 0.0);
            cudaEventRecord(e1, h->stream);
            if (!r && cudaEventSynchronize(e1) == cudaSuccess) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) t = std::min(t, ms);      // first run is a warm-up
            }
        }
        if (r) break;
        if (t < best) {
            best = t;
            pick = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    apply(pick);
    drop_graphs(h);
    if (r) return r;
    h->tuned = true;
    if (cache_path) {
        FILE* f = fopen(cache_path, "a");
        if (f) {
            fprintf(f, "%s=%d,%d,%d,%d\n", key, pick.variant, pick.threads, pick.grid, pick.f64t);
            fclose(f);
        }
    }
    return GAMER_OK;
}

int gamer_hydro_get_config(gamer_hydro_t h, char* buf, int len) {
    if (!h || !buf || len <= 0) return GAMER_ERR_ARG;
    snprintf(buf, (size_t)len, "%s kernel=%s threads=%d grid=%s fp64_threads=%d tuned=%d",
             h->precision == GAMER_FP32 ? "fp32" : "fp64", h->f32_variant == 0 ? "pipelined" : "simple",
             h->sweep_threads, h->grid_mode == 0 ? "one-per-SM" : "balanced", h->f64_threads, h->tuned ? 1 : 0);
    return GAMER_OK;
}

int gamer_hydro_set_profiling(gamer_hydro_t h, void* ev_before, void* ev_after) {
    if (!h) return GAMER_ERR_ARG;
    if ((ev_before == nullptr) != (ev_after == nullptr))
        return fail(h, GAMER_ERR_ARG, "give both events or neither");
    h->prof_ev[0] = static_cast<cudaEvent_t>(ev_before);
    h->prof_ev[1] = static_cast<cudaEvent_t>(ev_after);
    drop_graphs(h);
    return GAMER_OK;
}

const char* gamer_hydro_last_error(gamer_hydro_t h) {
    if (!h) return g_create_error.c_str();
    return h->err.c_str();
}

}  // extern "C"
