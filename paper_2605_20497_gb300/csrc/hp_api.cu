// hp_api.cu -- the multilevel driver (Sec. III) and the C ABI of include/hp.h.
//
// Coarsen level by level until ceil(|N|/Omega) nodes remain, no pair forms
// or max_levels is reached; the coarsest nodes are the initial parts; then
// project rho back level by level and refine every level (Sec. III, VI).
// Host control reads one counter per step; all arithmetic runs on the GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "hp_internal.cuh"

namespace hp {

static thread_local std::string t_last_error;

static int grid_of(int64_t n, int block) {
    int64_t g = cdiv(n, block);
    int64_t cap = (int64_t)num_sms() * 32;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}
#define GRID_STRIDE(i, n) \
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

__global__ void k_project(const int32_t *gamma, const int32_t *rho_coarse, int32_t n, int32_t *rho) {
    HP_KERNEL_ENTER();
    GRID_STRIDE(v, (int64_t)n) rho[v] = rho_coarse[gamma[v]];
}
__global__ void k_used(const int32_t *rho, int32_t n, int32_t *used) {
    HP_KERNEL_ENTER();
    GRID_STRIDE(v, (int64_t)n) used[rho[v]] = 1;
}
__global__ void k_compact_ids(const int32_t *rho, const int32_t *newid, int32_t n, int32_t *part) {
    HP_KERNEL_ENTER();
    GRID_STRIDE(v, (int64_t)n) part[v] = newid[rho[v]];
}
__global__ void k_check_parts(const int32_t *part, int32_t n, int32_t nparts, uint32_t *err) {
    HP_KERNEL_ENTER();
    GRID_STRIDE(v, (int64_t)n) {
        if (part[v] < 0 || part[v] >= nparts) atomicOr(err, E_INTERNAL);
    }
}

static hp_status status_of(uint32_t err) {
    if (err & (E_OFFSETS | E_PIN | E_SRC | E_DUP)) return HP_ERR_BAD_CSR;
    if (err & (E_WEIGHT | E_WSUM)) return HP_ERR_INVALID_ARG;
    if (err & E_INFEAS) return HP_ERR_INFEASIBLE;
    if (err & E_TIMEOUT) return HP_ERR_TIMEOUT;
    if (err & E_INTERNAL) return HP_ERR_INTERNAL;
    return HP_OK;
}

static bool options_ok(const hp_options &o) {
    if (o.pi < 1 || o.pi > 16 || o.theta < 0 || o.theta > 1024 || o.chain_window < 1 || o.chain_rounds < 0 ||
        o.chain_rounds > 1024 || o.noise_permille < 0 || o.noise_permille > 1000 ||
        (o.count_kind != HP_COUNT_INBOUND && o.count_kind != HP_COUNT_INCIDENT) || o.max_levels < 0 ||
        o.max_levels > 4096)
        return false;
    if (o.debug_walk_cap < 0 || o.node_batch < 0 || o.learned_levels < 0) return false;
    if (o.debug_table_cap != 0) {
        int c = o.debug_table_cap;
        if (c < 64 || c > 65536 || (c & (c - 1))) return false;
    }
    if (o.learned_k != 0 &&
        (o.learned_k < o.pi || o.learned_k > 16 || !o.merge_model || !merge_model_ok(*o.merge_model)))
        return false;
    return true;
}

// releases the level workspaces (streams, events, device memory) when a
// call ends early with an exception
struct WsGuard {
    Arena &A;
    CoarsenWs *cw = nullptr;
    LevelWs *rw = nullptr;
    explicit WsGuard(Arena &a) : A(a) {}
    ~WsGuard() {
        coarsen_workspace_free(cw, A);
        refine_workspace_free(rw, A);
    }
};

struct Timer {
    cudaEvent_t a, b, c, p[2];
    cudaStream_t s;
    explicit Timer(cudaStream_t st) : s(st) {
        HPC(cudaEventCreate(&a));
        HPC(cudaEventCreate(&b));
        HPC(cudaEventCreate(&c));
        HPC(cudaEventCreate(&p[0]));
        HPC(cudaEventCreate(&p[1]));
    }
    ~Timer() {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        cudaEventDestroy(c);
        cudaEventDestroy(p[0]);
        cudaEventDestroy(p[1]);
    }
};

static hp_status run(const int32_t *pins, const int32_t *offsets, int32_t e, int32_t n, const int32_t *src_counts,
                     const int32_t *weights, int32_t omega, int32_t delta, uint64_t seed, const hp_options *opt,
                     int32_t *part_out, hp_stats *stats, hp_level_trace *trace, int32_t trace_cap, cudaStream_t s) {
    Params P;
    P.omega = omega;
    P.delta = delta;
    P.seed = seed;
    if (opt) P.o = *opt;
    else hp_default_options(&P.o);
    if (n < 0 || e < 0 || omega < 1 || delta < 0 || !offsets || (n > 0 && !part_out) || !options_ok(P.o) ||
        (trace_cap > 0 && !trace))
        return HP_ERR_INVALID_ARG;
    noalloc_prepare();
    Timer T(s);
    const int64_t launches0 = t_launches;
    HPC(cudaEventRecord(T.a, s));
    Arena A(s);
    int32_t *w = A.get<int32_t>(e);
    std::vector<Level> lv(1);
    uint32_t err = validate_and_build_level0(pins, offsets, e, n, src_counts, weights, P, lv[0], w, A);
    if (err) return status_of(err);
    if (!pins && lv[0].np > 0) return HP_ERR_INVALID_ARG;
    hp_stats st;
    std::memset(&st, 0, sizeof st);
    std::vector<hp_level_trace> tr;
    if (n == 0) {
        if (stats) *stats = st;
        return HP_OK;
    }
    uint32_t *err_dev = A.get<uint32_t>(1);
    HPC(cudaMemsetAsync(err_dev, 0, sizeof(uint32_t), s));
    const int32_t max_e0 = max_edge_size(lv[0], A);

    // ---- coarsening (Sec. V)
    const int64_t target_n = ((int64_t)n + omega - 1) / omega;
    int32_t L = 0;
    bool prop0_timed = false;
    WsGuard guard(A);
    CoarsenWs *CW = guard.cw = coarsen_workspace(n, e, P, A);
    int32_t *mate = A.get<int32_t>(n);
    for (;;) {
        hp_level_trace t;
        std::memset(&t, 0, sizeof t);
        t.n = lv[L].n;
        t.pins = lv[L].np;
        if ((int64_t)lv[L].n <= target_n || L == P.o.max_levels) {
            tr.push_back(t);
            break;
        }
        PlainLaunchScope plain(lv[L].n > PDL_MAX_N);
        coarsen_level(lv[L], L, w, P, mate, *CW, A, err_dev, nullptr, nullptr, L == 0 ? T.p : nullptr);
        lv.emplace_back();
        LevelBox hb;
        const bool go = contract_level(lv[L], mate, coarsen_box(CW), &hb, lv[L + 1], A);
        if (hb.err) {
            // a bounded device loop of the level gave up: its matching is not
            // to be contracted
            t_last_error = "device check failed in coarsening level " + std::to_string(L) + " (error bits " +
                           std::to_string(hb.err) + ")";
            return status_of(hb.err);
        }
        st.pin_visits += (int64_t)hb.visits;
        {
            // algorithmic bytes of the level (see hp_stats.alg_bytes)
            const int64_t nl = lv[L].n, pl = lv[L].np, pi = P.o.pi;
            st.alg_bytes += 4 * (int64_t)hb.visits + 8 * (int64_t)hb.nbrs + 12 * pl + nl * (12 * pi + 4);
            st.alg_bytes += 48 * pi * nl;
            st.alg_bytes += 12 * pl + 16 * nl + (go ? 8 * (int64_t)hb.cnp : 0);
        }
        if (L == 0) {
            prop0_timed = true;
            st.l0_pin_visits = (int64_t)hb.visits;
            st.l0_neighbours = (int64_t)hb.nbrs;
        }
        t.pairs = (int32_t)(hb.pairs + hb.iso);
        t.iso_pairs = (int32_t)hb.iso;
        t.valid = t.n - hb.isolist;
        t.iso_list = hb.isolist;
        t.targets_r1 = hb.ntargets;
        t.max_indeg_r1 = hb.maxin;
        t.pairs_r1 = (int32_t)hb.pairs1;
        tr.push_back(t);
        if (!go) {
            lv.pop_back();
            break;
        }
        A.release(lv[L].nbnd);
        A.release(lv[L].pedge);
        lv[L].nbnd = lv[L].pedge = nullptr;
        L++;
    }
    coarsen_workspace_free(CW, A);
    guard.cw = nullptr;
    A.release(mate);
    HPC(cudaEventRecord(T.b, s));

    // ---- refinement (Sec. VI): coarsest clusters are the initial parts
    const int32_t nparts = lv[L].n;
    int32_t *rho = A.get<int32_t>(nparts);
    iota_i32(rho, nparts, s);
    int64_t *obj = A.get<int64_t>(2);
    LevelWs *RW = guard.rw = refine_workspace(lv[0].n, lv[0].np, lv[0].e, nparts, max_e0, P, A);
    for (int32_t l = L; l >= 0; l--) {
        Level &g = lv[l];
        if (l < L) {
            int32_t *r = A.get<int32_t>(g.n);
            launch_k(k_project, grid_of(g.n, 256), 256, 0, s, g.gamma, rho, g.n, r);
            HP_LAUNCH_CHECK();
            A.release(rho);
            rho = r;
            // the coarser level is no longer needed
            Level &c = lv[l + 1];
            for (int32_t *p : {c.off, c.pin, c.pedge, c.nsrc, c.size, c.ioff, c.inc, c.inode, c.nin, c.gamma, c.nbnd})
                A.release(p);
            c = Level();
        }
        PlainLaunchScope plain(g.n > PDL_MAX_N);
        RefineOut ro = refine_level(g, w, P, rho, RW, A, err_dev);
        st.moves_applied += ro.moves;
        st.alg_bytes += ro.alg_bytes;
        tr[l].reps = ro.reps;
        tr[l].moves = ro.moves;
        if (trace_cap > 0 && l < trace_cap) {
            objective(g, w, rho, nparts, obj, obj + 1, A);
            tr[l].conn = fetch<int64_t>(obj, s);
        }
    }
    refine_workspace_free(RW, A);
    guard.rw = nullptr;
    HPC(cudaEventRecord(T.c, s));

    // ---- compact part ids (ascending internal id) and statistics
    int32_t *used = A.get<int32_t>(nparts + 1);
    int32_t *newid = A.get<int32_t>(nparts + 1);
    HPC(cudaMemsetAsync(used, 0, sizeof(int32_t) * (nparts + 1), s));
    launch_k(k_used, grid_of(n, 256), 256, 0, s, rho, n, used);
    HP_LAUNCH_CHECK();
    scan_excl(used, newid, nparts, newid + nparts, A);
    const int32_t k = fetch<int32_t>(newid + nparts, s);
    int32_t *part = A.get<int32_t>(n);
    launch_k(k_compact_ids, grid_of(n, 256), 256, 0, s, rho, newid, n, part);
    HP_LAUNCH_CHECK();
    launch_k(k_check_parts, grid_of(n, 256), 256, 0, s, part, n, k, err_dev);
    HP_LAUNCH_CHECK();
    int64_t *ps = A.get<int64_t>(5);
    part_stats(lv[0], w, part, k, omega, delta, ps, A);
    int64_t hs[5];
    fetch_bytes(hs, ps, sizeof hs, s);
    uint32_t derr = fetch<uint32_t>(err_dev, s);
    if (derr) {
        t_last_error = "device check failed (error bits " + std::to_string(derr) + ")";
        return status_of(derr);
    }
    HPC(cudaMemcpyAsync(part_out, part, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    HPC(cudaStreamSynchronize(s));
    float ms_all = 0, ms_c = 0, ms_r = 0;
    HPC(cudaEventElapsedTime(&ms_all, T.a, T.c));
    HPC(cudaEventElapsedTime(&ms_c, T.a, T.b));
    HPC(cudaEventElapsedTime(&ms_r, T.b, T.c));
    if (prop0_timed) {
        float mp = 0;
        HPC(cudaEventElapsedTime(&mp, T.p[0], T.p[1]));
        st.ms_propose_l0 = mp;
    }
    st.kernel_launches = t_launches - launches0;
    st.connectivity = hs[0];
    st.cut_net = hs[1];
    st.num_parts = k;
    st.max_part_size = (int32_t)hs[2];
    st.max_part_distinct = (int32_t)hs[3];
    st.violations = (int32_t)hs[4];
    st.levels = L + 1;
    st.ms_total = ms_all;
    st.ms_coarsen = ms_c;
    st.ms_refine = ms_r;
    if (stats) *stats = st;
    for (int32_t l = 0; l < trace_cap && l < (int32_t)tr.size(); l++) trace[l] = tr[l];
    return HP_OK;
}

void set_last_error(const std::string &msg) { t_last_error = msg; }

template <class F> static hp_status guarded(F &&f) {
    try {
        t_last_error.clear();
        return f();
    } catch (const Error &x) {
        t_last_error = x.what();
        return x.status;
    } catch (const std::bad_alloc &) {
        t_last_error = "host allocation failed";
        return HP_ERR_OOM;
    } catch (const std::exception &x) {
        t_last_error = x.what();
        return HP_ERR_INTERNAL;
    }
}

}  // namespace hp

extern "C" {

void hp_default_options(hp_options *o) {
    if (!o) return;
    o->pi = 4;
    o->theta = 16;
    o->chain_window = 256;
    o->chain_rounds = 16;
    o->noise_permille = 100;
    o->count_kind = HP_COUNT_INBOUND;
    o->max_levels = 256;
    o->debug_table_cap = 0;
    o->learned_k = 0;
    o->debug_walk_cap = 0;
    o->merge_model = nullptr;
    o->node_batch = 0;
    o->learned_levels = 0;
}

hp_status hp_merge_features(const int32_t *pins, const int32_t *offsets, int32_t num_hedges, int32_t num_nodes,
                            const int32_t *src_counts, const int32_t *weights, int32_t omega, int32_t delta,
                            uint64_t seed, const hp_options *opt, int32_t *cand_out, int32_t *rank_out,
                            uint8_t *feat_out, void *stream) {
    return hp::guarded([&]() -> hp_status {
        if (!opt || num_nodes < 0 || num_hedges < 0 || omega < 1 || delta < 0 || !offsets) return HP_ERR_INVALID_ARG;
        hp::Params P;
        P.omega = omega;
        P.delta = delta;
        P.seed = seed;
        P.o = *opt;
        const int32_t K = P.o.learned_k;
        hp_options plain = P.o;   // every other option as hp_partition checks it
        plain.learned_k = 0;
        if (K < P.o.pi || K > 16 || !hp::options_ok(plain)) return HP_ERR_INVALID_ARG;
        if (num_nodes > 0 && (!cand_out || !rank_out || !feat_out || (reinterpret_cast<uintptr_t>(feat_out) & 15)))
            return HP_ERR_INVALID_ARG;
        P.o.merge_model = nullptr;
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        hp::Arena A(s);
        int32_t *w = A.get<int32_t>(num_hedges);
        hp::Level L;
        uint32_t err = hp::validate_and_build_level0(pins, offsets, num_hedges, num_nodes, src_counts, weights, P, L, w,
                                                     A);
        if (err) return hp::status_of(err);
        if (num_nodes == 0) return HP_OK;
        uint32_t *err_dev = A.get<uint32_t>(1);
        HPC(cudaMemsetAsync(err_dev, 0, sizeof(uint32_t), s));
        hp::CoarsenWs *CW = hp::coarsen_workspace(num_nodes, num_hedges, P, A);
        hp::level_features(L, w, P, *CW, A, err_dev, cand_out, rank_out, feat_out);
        hp::coarsen_workspace_free(CW, A);
        const uint32_t e = hp::fetch<uint32_t>(err_dev, s);
        if (e) return hp::status_of(e);
        HPC(cudaStreamSynchronize(s));
        return HP_OK;
    });
}

hp_status hp_merge_grad(const uint8_t *feat, const float *label, int64_t count, const float *params, float *grad_out,
                        double *loss_out, void *stream) {
    return hp::guarded([&]() -> hp_status {
        if (count < 0 || !params || !grad_out || (count > 0 && (!feat || !label))) return HP_ERR_INVALID_ARG;
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        hp::Arena A(s);
        const double loss = hp::merge_grad(feat, label, count, params, grad_out, A);
        if (loss_out) *loss_out = loss;
        HPC(cudaStreamSynchronize(s));
        return HP_OK;
    });
}

hp_status hp_merge_adam(float *params, const float *grad, float *m, float *v, int64_t step, float lr, float beta1,
                        float beta2, float eps, float weight_decay, void *stream) {
    return hp::guarded([&]() -> hp_status {
        if (!params || !grad || !m || !v || step < 1 || !(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) ||
            !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f) || !(weight_decay >= 0.f))
            return HP_ERR_INVALID_ARG;
        hp::merge_adam(params, grad, m, v, step, lr, beta1, beta2, eps, weight_decay,
                       static_cast<cudaStream_t>(stream));
        return HP_OK;
    });
}

hp_status hp_merge_quantize(const float *params, const uint8_t *calib, int64_t count, hp_merge_model *out) {
    return hp::guarded([&]() -> hp_status {
        if (!params || !calib || count < 1 || !out) return HP_ERR_INVALID_ARG;
        for (int i = 0; i < HP_MERGE_NPARAM; i++)
            if (!std::isfinite(params[i])) return HP_ERR_INVALID_ARG;
        hp_merge_model m;
        hp::merge_quantize(params, calib, count, m);
        *out = m;
        return HP_OK;
    });
}

hp_status hp_merge_scores(const uint8_t *feat, int64_t count, const hp_merge_model *model, int32_t *score_out,
                          void *stream) {
    return hp::guarded([&]() -> hp_status {
        if (count < 0 || !model || (count > 0 && (!feat || !score_out)) || !hp::merge_model_ok(*model))
            return HP_ERR_INVALID_ARG;
        if (count == 0) return HP_OK;
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        hp::Arena A(s);
        hp_merge_model *dm = A.get<hp_merge_model>(1);
        HPC(cudaMemcpyAsync(dm, model, sizeof(hp_merge_model), cudaMemcpyHostToDevice, s));
        hp::merge_scores(feat, count, dm, score_out, s);
        HPC(cudaStreamSynchronize(s));
        return HP_OK;
    });
}

hp_status hp_partition_ex(const int32_t *pins, const int32_t *offsets, int32_t num_hedges, int32_t num_nodes,
                          const int32_t *src_counts, const int32_t *weights, int32_t omega, int32_t delta,
                          uint64_t seed, const hp_options *opt, int32_t *part_out, hp_stats *stats,
                          hp_level_trace *trace, int32_t trace_cap, void *stream) {
    return hp::guarded([&] {
        return hp::run(pins, offsets, num_hedges, num_nodes, src_counts, weights, omega, delta, seed, opt, part_out,
                       stats, trace, trace_cap, static_cast<cudaStream_t>(stream));
    });
}

hp_status hp_partition(const int32_t *pins, const int32_t *offsets, int32_t num_hedges, int32_t num_nodes,
                       const int32_t *src_counts, const int32_t *weights, int32_t omega, int32_t delta, uint64_t seed,
                       const hp_options *opt, int32_t *part_out, hp_stats *stats, void *stream) {
    return hp_partition_ex(pins, offsets, num_hedges, num_nodes, src_counts, weights, omega, delta, seed, opt,
                           part_out, stats, nullptr, 0, stream);
}

hp_status hp_partition_host(const int32_t *pins, const int32_t *offsets, int32_t num_hedges, int32_t num_nodes,
                            const int32_t *src_counts, const int32_t *weights, int32_t omega, int32_t delta,
                            uint64_t seed, const hp_options *opt, int32_t *part_out, hp_stats *stats, void *stream) {
    return hp::guarded([&]() -> hp_status {
        if (num_hedges < 0 || num_nodes < 0 || !offsets || (num_nodes > 0 && !part_out)) return HP_ERR_INVALID_ARG;
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        hp::Arena A(s);
        const int64_t np = offsets[num_hedges];
        if (np < 0 || (np > 0 && !pins)) return HP_ERR_BAD_CSR;
        int32_t *d_off = A.get<int32_t>(num_hedges + 1);
        int32_t *d_pins = A.get<int32_t>(np);
        int32_t *d_src = src_counts ? A.get<int32_t>(num_hedges) : nullptr;
        int32_t *d_w = weights ? A.get<int32_t>(num_hedges) : nullptr;
        int32_t *d_part = A.get<int32_t>(num_nodes);
        HPC(cudaMemcpyAsync(d_off, offsets, sizeof(int32_t) * (num_hedges + 1), cudaMemcpyHostToDevice, s));
        if (np) HPC(cudaMemcpyAsync(d_pins, pins, sizeof(int32_t) * np, cudaMemcpyHostToDevice, s));
        if (d_src) HPC(cudaMemcpyAsync(d_src, src_counts, sizeof(int32_t) * num_hedges, cudaMemcpyHostToDevice, s));
        if (d_w) HPC(cudaMemcpyAsync(d_w, weights, sizeof(int32_t) * num_hedges, cudaMemcpyHostToDevice, s));
        hp_status r = hp::run(d_pins, d_off, num_hedges, num_nodes, d_src, d_w, omega, delta, seed, opt, d_part, stats,
                              nullptr, 0, s);
        if (r != HP_OK) return r;
        if (num_nodes) HPC(cudaMemcpyAsync(part_out, d_part, sizeof(int32_t) * num_nodes, cudaMemcpyDeviceToHost, s));
        HPC(cudaStreamSynchronize(s));
        return HP_OK;
    });
}

hp_status hp_set_allocator(void *(*alloc_fn)(size_t, void *), void (*free_fn)(void *, void *), void *ctx) {
    if ((alloc_fn == nullptr) != (free_fn == nullptr)) return HP_ERR_INVALID_ARG;
    hp::set_allocator(alloc_fn, free_fn, ctx);
    return HP_OK;
}

const char *hp_status_string(hp_status s) {
    switch (s) {
    case HP_OK: return "ok";
    case HP_ERR_INVALID_ARG: return "invalid argument";
    case HP_ERR_BAD_CSR: return "malformed CSR hypergraph";
    case HP_ERR_INFEASIBLE: return "infeasible: a node alone exceeds Delta";
    case HP_ERR_OOM: return "out of device memory";
    case HP_ERR_CUDA: return "CUDA error";
    case HP_ERR_TIMEOUT: return "bounded device loop ran out of iterations";
    case HP_ERR_INTERNAL: return "internal error";
    }
    return "unknown status";
}

const char *hp_last_error(void) { return hp::t_last_error.c_str(); }

hp_status hp_connectivity(const int32_t *pins, const int32_t *offsets, int32_t num_hedges, const int32_t *weights,
                          const int32_t *part, int32_t num_nodes, int32_t num_parts, int64_t *conn_out,
                          int64_t *cutnet_out, void *stream) {
    return hp::guarded([&]() -> hp_status {
        if (num_hedges < 0 || num_nodes < 0 || num_parts < 0 || !offsets || (num_nodes > 0 && !part))
            return HP_ERR_INVALID_ARG;
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        hp::noalloc_prepare();
        hp::Arena A(s);
        hp::Params P;
        P.omega = 1;
        P.delta = 0x7fffffff;
        P.seed = 0;
        hp_default_options(&P.o);
        hp::Level L;
        int32_t *w = A.get<int32_t>(num_hedges);
        uint32_t err = hp::validate_and_build_level0(pins, offsets, num_hedges, num_nodes, nullptr, weights, P, L, w, A);
        if (err) return hp::status_of(err);
        uint32_t *e2 = A.get<uint32_t>(1);
        HPC(cudaMemsetAsync(e2, 0, sizeof(uint32_t), s));
        if (num_nodes > 0) {
            hp::launch_k(hp::k_check_parts, hp::grid_of(num_nodes, 256), 256, 0, s, part, num_nodes, num_parts, e2);
            HP_LAUNCH_CHECK();
        }
        if (hp::fetch<uint32_t>(e2, s)) return HP_ERR_INVALID_ARG;
        int64_t *obj = A.get<int64_t>(2);
        hp::objective(L, w, part, num_parts, obj, obj + 1, A);
        int64_t h[2];
        hp::fetch_bytes(h, obj, sizeof h, s);
        if (conn_out) *conn_out = h[0];
        if (cutnet_out) *cutnet_out = h[1];
        return HP_OK;
    });
}

hp_status hp_debug_coarsen_level(int32_t num_nodes, int32_t num_hedges, const int32_t *offsets, const int32_t *pins,
                                 const int32_t *src_counts, const int32_t *weights, const int32_t *size, int32_t omega,
                                 int32_t delta, uint64_t seed, int32_t level, const hp_options *opt, int32_t *cand_out,
                                 uint64_t *score_out, int32_t *mate_out, int64_t *pairs_out, void *stream) {
    return hp::guarded([&]() -> hp_status {
        hp::Params P;
        P.omega = omega;
        P.delta = delta;
        P.seed = seed;
        if (opt) P.o = *opt;
        else hp_default_options(&P.o);
        if (num_nodes < 1 || num_hedges < 0 || omega < 1 || delta < 0 || level < 0 || !offsets || !src_counts ||
            !weights || !size || !cand_out || !score_out || !mate_out || !hp::options_ok(P.o))
            return HP_ERR_INVALID_ARG;
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        hp::Arena A(s);
        hp::Level L;
        hp::make_level(num_nodes, num_hedges, offsets, pins, src_counts, size, L, A);
        uint32_t *err = A.get<uint32_t>(1);
        HPC(cudaMemsetAsync(err, 0, sizeof(uint32_t), s));
        hp::CoarsenWs *CW = hp::coarsen_workspace(num_nodes, num_hedges, P, A);
        hp::coarsen_level(L, level, weights, P, mate_out, *CW, A, err, cand_out, score_out);
        hp::LevelBox hb;
        hp::fetch_bytes(&hb, hp::coarsen_box(CW), sizeof hb, s);
        hp::coarsen_workspace_free(CW, A);
        uint32_t e = hp::fetch<uint32_t>(err, s);
        if (e) return hp::status_of(e);
        if (pairs_out) *pairs_out = (int64_t)(hb.pairs + hb.iso);
        return HP_OK;
    });
}

hp_status hp_debug_refine_rep(int32_t num_nodes, int32_t num_hedges, const int32_t *offsets, const int32_t *pins,
                              const int32_t *src_counts, const int32_t *weights, const int32_t *size, int32_t *rho,
                              int32_t num_parts, int32_t second_half, int32_t omega, int32_t delta,
                              const hp_options *opt, int32_t *move_node, int32_t *move_src, int32_t *move_dst,
                              int64_t *move_gain, int32_t *seq, int64_t *gseq, int32_t *num_moves, int32_t *applied,
                              int64_t *best_gain, void *stream) {
    return hp::guarded([&]() -> hp_status {
        hp::Params P;
        P.omega = omega;
        P.delta = delta;
        P.seed = 0;
        if (opt) P.o = *opt;
        else hp_default_options(&P.o);
        if (num_nodes < 1 || num_hedges < 0 || num_parts < 1 || omega < 1 || delta < 0 || !offsets ||
            !src_counts || !weights || !size || !rho || !move_node || !move_src || !move_dst || !move_gain ||
            !seq || !gseq || !hp::options_ok(P.o))
            return HP_ERR_INVALID_ARG;
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        hp::Arena A(s);
        hp::Level L;
        hp::make_level(num_nodes, num_hedges, offsets, pins, src_counts, size, L, A);
        P.wsum = (int64_t)num_hedges * 65536;
        uint32_t *err = A.get<uint32_t>(1);
        long long *bg = A.get<long long>(1);
        HPC(cudaMemsetAsync(err, 0, sizeof(uint32_t), s));
        HPC(cudaMemsetAsync(bg, 0, sizeof(long long), s));
        int32_t m = 0;
        hp::RepDebug D{move_node, move_src, move_dst, reinterpret_cast<long long *>(move_gain), seq,
                       reinterpret_cast<long long *>(gseq), bg, &m};
        int32_t k = hp::refine_rep_debug(L, weights, num_parts, P, rho, second_half, A, err, D);
        uint32_t e = hp::fetch<uint32_t>(err, s);
        if (e) return hp::status_of(e);
        if (num_moves) *num_moves = m;
        if (applied) *applied = k;
        if (best_gain) *best_gain = hp::fetch<long long>(bg, s);
        return HP_OK;
    });
}

}  // extern "C"
