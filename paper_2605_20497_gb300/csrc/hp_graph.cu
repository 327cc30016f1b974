// hp_graph.cu -- input checks, incidence sets (Sec. IV-B) and coarse
// hypergraph construction (Sec. V-E).
#include <cuda_runtime.h>

#include "hp_cluster.cuh"
#include "hp_internal.cuh"

namespace hp {

static int grid_of(int64_t n, int block) {
    int64_t g = cdiv(n, block);
    int64_t cap = (int64_t)num_sms() * 32;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}
#define GRID_STRIDE(i, n) \
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)
#define CSTRIDE_G(i, n, t0, nt) for (int64_t i = (t0); i < (int64_t)(n); i += (nt))

// ---------------------------------------------------------------- checks
__global__ void k_check_offsets(const int32_t *off, int32_t e, uint32_t *err) {
    HP_KERNEL_ENTER();
    GRID_STRIDE(i, (int64_t)e) {
        if (off[i + 1] <= off[i]) atomicOr(err, E_OFFSETS);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && off[0] != 0) atomicOr(err, E_OFFSETS);
}

__global__ void k_edges_level0(const int32_t *off, int32_t e, const int32_t *src_counts, const int32_t *weights,
                               int32_t kind, int32_t *nsrc, int32_t *w, unsigned long long *wsum, uint32_t *err) {
    HP_KERNEL_ENTER();
    GRID_STRIDE(i, (int64_t)e) {
        int32_t sz = off[i + 1] - off[i];
        int32_t s = src_counts ? src_counts[i] : 1;
        if (s < 0 || s > sz) atomicOr(err, E_SRC);
        nsrc[i] = kind == HP_COUNT_INCIDENT ? 0 : s;
        int32_t wi = weights ? weights[i] : 1;
        if (wi < 1 || wi > 65536) atomicOr(err, E_WEIGHT);
        w[i] = wi;
        if (weights) atomicAdd(wsum, (unsigned long long)(wi < 0 ? 0 : wi));
    }
}

// pedge[j] = hyperedge of pin position j (one warp per hyperedge)
__global__ void k_pin_edges(const int32_t *off, int32_t e, int32_t *pedge) {
    HP_KERNEL_ENTER();
    int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < e; i += nw)
        for (int32_t j = off[i] + lane; j < off[i + 1]; j += 32) pedge[j] = (int32_t)i;
}

__global__ void k_check_pins(const int32_t *pin, int64_t np, int32_t n, uint32_t *err) {
    HP_KERNEL_ENTER();
    GRID_STRIDE(j, np) {
        int32_t v = pin[j];
        if (v < 0 || v >= n) atomicOr(err, E_PIN);
    }
}

// duplicates: an edge twice in in(v) or out(v), or in both (src & dst overlap)
__global__ void k_check_dups(const int32_t *ioff, const int32_t *inc, const int32_t *nin, int32_t n, int32_t delta,
                             uint32_t *err) {
    HP_KERNEL_ENTER();
    GRID_STRIDE(v, (int64_t)n) {
        int32_t a = ioff[v], m = a + nin[v], b = ioff[v + 1];
        bool dup = false;
        for (int32_t t = a + 1; t < b && !dup; t++)
            if (t != m && inc[t] == inc[t - 1]) dup = true;
        for (int32_t t = m; t < b && !dup; t++) {
            int32_t x = inc[t], lo = a, hi = m;
            while (lo < hi) {
                int32_t mid = (lo + hi) >> 1;
                if (inc[mid] < x) lo = mid + 1;
                else hi = mid;
            }
            if (lo < m && inc[lo] == x) dup = true;
        }
        if (dup) atomicOr(err, E_DUP);
        if (nin[v] > delta) atomicOr(err, E_INFEAS);
    }
}

// ---------------------------------------------------------------- incidence
// counts per node are combined across the lanes holding the same node
// before the atomics (hub nodes appear in many hyperedges of a warp)
__global__ void k_inc_keys(const int32_t *pin, const int32_t *pedge, const int32_t *off, const int32_t *nsrc,
                           int64_t np, uint32_t *keys, uint32_t *vals, int32_t *cnt, int32_t *nin) {
    HP_KERNEL_ENTER();
    const int lane = threadIdx.x & 31;
    const int64_t wbase = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) << 5;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = wbase; base < np; base += stride) {
        const int64_t j = base + lane;
        const bool valid = j < np;
        int32_t v = -1 - lane;
        bool src = false;
        if (valid) {
            const int32_t e = pedge[j];
            v = pin[j];
            src = (int32_t)j - off[e] < nsrc[e];
            keys[j] = (uint32_t)v * 2u + (src ? 1u : 0u);
            vals[j] = (uint32_t)e;
        }
        const uint32_t peers = __match_any_sync(0xffffffffu, v);
        const uint32_t dstpeers = __ballot_sync(0xffffffffu, valid && !src) & peers;
        if (valid && lane == __ffs(peers) - 1) {
            atomicAdd(&cnt[v], __popc(peers));
            if (dstpeers) atomicAdd(&nin[v], __popc(dstpeers));
        }
    }
}

__global__ void k_inc_nodes(const uint32_t *keys, int64_t np, int32_t *inode) {
    HP_KERNEL_ENTER();
    GRID_STRIDE(j, np) inode[j] = (int32_t)(keys[j] >> 1);
}

void build_incidence(Level &L, Arena &A) {
    cudaStream_t s = A.stream();
    L.ioff = A.get<int32_t>(L.n + 1);
    L.nin = A.get<int32_t>(L.n);
    L.inc = A.get<int32_t>(L.np);
    int32_t *cnt = A.get<int32_t>(L.n + 1);
    HPC(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (L.n + 1), s));
    HPC(cudaMemsetAsync(L.nin, 0, sizeof(int32_t) * L.n, s));
    uint32_t *keys = A.get<uint32_t>(L.np);
    if (L.np > 0) {
        launch_k(k_inc_keys, grid_of(L.np, 256), 256, 0, s, L.pin, L.pedge, L.off, L.nsrc, L.np, keys,
                 reinterpret_cast<uint32_t *>(L.inc), cnt, L.nin);
        HP_LAUNCH_CHECK();
        radix_sort(keys, reinterpret_cast<uint32_t *>(L.inc), L.np, bits_for(2ull * (uint64_t)L.n - 1), A);
    }
    scan_excl(cnt, L.ioff, L.n + 1, nullptr, A);
    L.inode = A.get<int32_t>(L.np);
    if (L.np > 0) {
        launch_k(k_inc_nodes, grid_of(L.np, 256), 256, 0, s, keys, L.np, L.inode);
        HP_LAUNCH_CHECK();
    }
    A.release(keys);
    A.release(cnt);
}

uint32_t validate_and_build_level0(const int32_t *pins, const int32_t *offsets, int32_t e, int32_t n,
                                   const int32_t *src_counts, const int32_t *weights, Params &P, Level &L,
                                   int32_t *w, Arena &A) {
    cudaStream_t s = A.stream();
    struct Box {
        uint32_t err, pad;
        unsigned long long wsum;
        int32_t np;
    };
    Box *box = A.get<Box>(1);
    HPC(cudaMemsetAsync(box, 0, sizeof(Box), s));
    if (e > 0) {
        launch_k(k_check_offsets, grid_of(e, 256), 256, 0, s, offsets, e, &box->err);
        HP_LAUNCH_CHECK();
        HPC(cudaMemcpyAsync(&box->np, offsets + e, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    } else {
        // no hyperedges: offsets[0] must still be 0
        HPC(cudaMemcpyAsync(&box->np, offsets, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    }
    Box hb;
    fetch_bytes(&hb, box, sizeof(Box), s);
    if (e == 0 && hb.np != 0) hb.err |= E_OFFSETS;
    if (hb.err) return hb.err;
    L.n = n;
    L.e = e;
    L.np = hb.np;
    L.off = A.get<int32_t>(e + 1);
    HPC(cudaMemcpyAsync(L.off, offsets, sizeof(int32_t) * (e + 1), cudaMemcpyDeviceToDevice, s));
    L.pin = A.get<int32_t>(L.np);
    if (L.np) HPC(cudaMemcpyAsync(L.pin, pins, sizeof(int32_t) * L.np, cudaMemcpyDeviceToDevice, s));
    L.nsrc = A.get<int32_t>(e);
    L.pedge = A.get<int32_t>(L.np);
    if (e > 0) {
        launch_k(k_edges_level0, grid_of(e, 256), 256, 0, s, L.off, e, src_counts, weights, P.o.count_kind, L.nsrc, w,
                 &box->wsum, &box->err);
        HP_LAUNCH_CHECK();
        launch_k(k_pin_edges, grid_of((int64_t)e * 32, 256), 256, 0, s, L.off, e, L.pedge);
        HP_LAUNCH_CHECK();
    }
    if (L.np) {
        launch_k(k_check_pins, grid_of(L.np, 256), 256, 0, s, L.pin, L.np, n, &box->err);
        HP_LAUNCH_CHECK();
    }
    fetch_bytes(&hb, box, sizeof(Box), s);
    if (hb.wsum > (1ull << 37)) hb.err |= E_WSUM;
    if (hb.err & (E_PIN | E_SRC)) return hb.err;
    build_incidence(L, A);
    if (n > 0) {
        launch_k(k_check_dups, grid_of(n, 256), 256, 0, s, L.ioff, L.inc, L.nin, n, P.delta, &box->err);
        HP_LAUNCH_CHECK();
    }
    L.size = A.get<int32_t>(n);
    fill_i32(L.size, n, 1, s);
    L.nbnd = A.get<int32_t>(n);
    fill_i32(L.nbnd, n, n > 0 ? n - 1 : 0, s);
    fetch_bytes(&hb, box, sizeof(Box), s);
    if (hb.wsum > (1ull << 37)) hb.err |= E_WSUM;
    P.wsum = weights ? (int64_t)hb.wsum : (int64_t)e;
    A.release(box);
    return hb.err;
}

void make_level(int32_t n, int32_t e, const int32_t *off, const int32_t *pins, const int32_t *nsrc,
                const int32_t *size, Level &L, Arena &A) {
    cudaStream_t s = A.stream();
    L.n = n;
    L.e = e;
    L.off = A.get<int32_t>(e + 1);
    HPC(cudaMemcpyAsync(L.off, off, sizeof(int32_t) * (e + 1), cudaMemcpyDeviceToDevice, s));
    L.np = fetch<int32_t>(L.off + e, s);
    L.pin = A.get<int32_t>(L.np);
    if (L.np) HPC(cudaMemcpyAsync(L.pin, pins, sizeof(int32_t) * L.np, cudaMemcpyDeviceToDevice, s));
    L.nsrc = A.get<int32_t>(e);
    if (e) HPC(cudaMemcpyAsync(L.nsrc, nsrc, sizeof(int32_t) * e, cudaMemcpyDeviceToDevice, s));
    L.size = A.get<int32_t>(n);
    if (n) HPC(cudaMemcpyAsync(L.size, size, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    L.pedge = A.get<int32_t>(L.np);
    if (e > 0) {
        launch_k(k_pin_edges, grid_of((int64_t)e * 32, 256), 256, 0, s, L.off, e, L.pedge);
        HP_LAUNCH_CHECK();
    }
    build_incidence(L, A);
    L.nbnd = A.get<int32_t>(n);
    fill_i32(L.nbnd, n, n > 0 ? n - 1 : 0, s);
}

// ---------------------------------------------------------------- contraction
__device__ __forceinline__ int32_t lower_bound_seg(const int32_t *a, int32_t lo, int32_t hi, int32_t x) {
    while (lo < hi) {
        int32_t mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Keep rule realising dst' = gamma(dst(e)), src' = gamma(src(e)) \ dst' with
// one copy per cluster: a pin whose partner is not in e is kept; two
// destinations (or two sources) keep the smaller id; a source whose partner
// is a destination of e is dropped (the cluster is in dst').
__device__ __forceinline__ int32_t pin_keep(const int32_t *pin, const int32_t *pedge, const int32_t *off,
                                            const int32_t *nsrc, const int32_t *mate, const int32_t *ioff,
                                            const int32_t *inc, const int32_t *nin, int64_t j) {
    int32_t e = pedge[j], p = pin[j];
    bool p_src = (int32_t)j - off[e] < nsrc[e];
    int32_t q = mate[p];
    int k = 1;
    if (q >= 0) {
        int32_t a = ioff[q], m = a + nin[q], b = ioff[q + 1];
        int32_t t = lower_bound_seg(inc, a, m, e);
        bool q_dst = t < m && inc[t] == e;
        bool q_src = false;
        if (!q_dst) {
            t = lower_bound_seg(inc, m, b, e);
            q_src = t < b && inc[t] == e;
        }
        if (p_src) k = (!q_dst && !q_src) || (q_src && p < q);
        else k = (!q_dst && !q_src) || q_src || p < q;
    }
    return k;
}



// ---------------------------------------------------------------- coarse incidence by rank
// The coarse incidence is not sorted anew.  A coarse node c = {u, w} has
// in(c) = in(u) U in(w) and out(c) = (out(u) U out(w)) \ in(c), each
// ascending by hyperedge, and an incidence entry (v, e) survives exactly when
// the pin v of e survives (the keep rule above, seen from the node's side).
// So every surviving entry of u or w is written straight to its place: its
// rank among the surviving entries of its own list plus the number of
// surviving entries of the partner's list below it (one binary search), both
// read off one prefix sum over the keep flags of the fine incidence.
// Levels of up to CONTRACT_CLUSTER_NP pins run the steps in one launch on one
// thread-block cluster; larger ones as a few grid-wide kernels.
constexpr int64_t CONTRACT_CLUSTER_NP = int64_t(1) << 15;

struct ContractArgs {
    Level L;                 // the fine level
    const int32_t *mate;
    LevelBox *box;           // cn, cnp are written here
    int32_t *isrep, *cid, *rep_of, *ccnt;   // scratch of n entries
    // per fine pin position / incidence entry: (pin survives) << 32 | (entry
    // survives), and its exclusive prefix sum (np + 1 entries): the high
    // words number the coarse pins, the low words the coarse incidence
    int64_t *kflag, *kscan;
    Level C;                 // coarse arrays allocated for L.n nodes and L.np pins (ioff: n + 1)
    int32_t *gamma;          // [L.n]
};

__device__ __forceinline__ bool in_sorted(const int32_t *a, int32_t lo, int32_t hi, int32_t x) {
    const int32_t t = lower_bound_seg(a, lo, hi, x);
    return t < hi && a[t] == x;
}

// whether incidence entry t of the fine level survives contraction: the
// entry (v, e) of a destination survives unless v is the larger member of
// its pair and the partner is also a destination of e; the entry of a
// source survives unless the partner is a destination of e, or v is the
// larger member and the partner is also a source of e
__device__ __forceinline__ int32_t inc_keep(const Level &L, const int32_t *mate, int64_t t) {
    const int32_t v = L.inode[t], w = mate[v];
    if (w < 0) return 1;
    const int32_t e = L.inc[t];
    const int32_t wa = L.ioff[w], wm = wa + L.nin[w], wb = L.ioff[w + 1];
    const bool w_dst = in_sorted(L.inc, wa, wm, e);
    if (t < (int64_t)L.ioff[v] + L.nin[v]) return (v < w || !w_dst) ? 1 : 0;
    if (w_dst) return 0;
    return (v < w || !in_sorted(L.inc, wm, wb, e)) ? 1 : 0;
}

__device__ __forceinline__ int32_t newpos_of(const ContractArgs &A, int64_t j) { return (int32_t)(A.kscan[j] >> 32); }
__device__ __forceinline__ int32_t ipos_of(const ContractArgs &A, int64_t t) { return (int32_t)(uint32_t)A.kscan[t]; }

// a level whose matching formed no pair is not contracted; one whose
// matching gave up is reported by the host and not contracted either
__device__ __forceinline__ bool contract_off(const LevelBox *box) {
    return box->err != 0u || box->pairs + box->iso == 0ull;
}

// representatives (the smaller member of a pair), surviving pins and
// surviving incidence entries
__device__ __forceinline__ void ph_c_flags(const ContractArgs &A, int64_t t0, int64_t nt) {
    const Level &L = A.L;
    CSTRIDE_G(v, L.n, t0, nt) {
        const int32_t m = A.mate[v];
        A.isrep[v] = (m < 0 || (int32_t)v < m) ? 1 : 0;
    }
    CSTRIDE_G(j, L.np, t0, nt)
        A.kflag[j] = ((int64_t)pin_keep(L.pin, L.pedge, L.off, L.nsrc, A.mate, L.ioff, L.inc, L.nin, j) << 32) |
                     (int64_t)inc_keep(L, A.mate, j);
}

// gamma, coarse sizes and neighbour bounds, the representative of every
// coarse node, coarse hyperedge segments
__device__ __forceinline__ void ph_c_map(const ContractArgs &A, int64_t t0, int64_t nt) {
    const Level &L = A.L;
    const Level &C = A.C;
    const int32_t cnp = newpos_of(A, L.np);
    CSTRIDE_G(v0, L.n, t0, nt) {
        const int32_t v = (int32_t)v0, m = A.mate[v];
        const int32_t r = (m >= 0 && m < v) ? m : v, g = A.cid[r];
        A.gamma[v] = g;
        if (r == v) {
            C.size[g] = L.size[v] + (m >= 0 ? L.size[m] : 0);
            const int64_t b = (int64_t)L.nbnd[v] + (m >= 0 ? L.nbnd[m] : 0);
            C.nbnd[g] = b > 0x7fffffff ? 0x7fffffff : (int32_t)b;
            A.rep_of[g] = v;
        }
    }
    CSTRIDE_G(i, L.e, t0, nt) {
        const int32_t a = newpos_of(A, L.off[i]);
        C.off[i] = a;
        C.nsrc[i] = newpos_of(A, (int64_t)L.off[i] + L.nsrc[i]) - a;
    }
    if (t0 == 0) {
        C.off[L.e] = cnp;
        A.box->cnp = cnp;
    }
}

// coarse pins; surviving incidence entries per coarse node (0 beyond the
// last coarse node, so that a scan over L.n entries ends every segment)
__device__ __forceinline__ void ph_c_pins(const ContractArgs &A, int64_t t0, int64_t nt) {
    const Level &L = A.L;
    const Level &C = A.C;
    const int32_t cn = A.box->cn;
    CSTRIDE_G(j, L.np, t0, nt) {
        if (A.kflag[j] >> 32) {
            const int32_t k = newpos_of(A, j);
            C.pin[k] = A.gamma[L.pin[j]];
            C.pedge[k] = L.pedge[j];
        }
    }
    CSTRIDE_G(c, L.n, t0, nt) {
        int32_t kd = 0, ks = 0;
        if (c < cn) {
            const int32_t u = A.rep_of[c], w = A.mate[u];
            for (int k = 0; k < 2; k++) {
                const int32_t v = k == 0 ? u : w;
                if (v < 0) break;
                const int32_t a = L.ioff[v], m = a + L.nin[v], b = L.ioff[v + 1];
                kd += ipos_of(A, m) - ipos_of(A, a);
                ks += ipos_of(A, b) - ipos_of(A, m);
            }
            C.nin[c] = kd;
        }
        A.ccnt[c] = kd + ks;
    }
}

// every surviving incidence entry at its rank in the coarse lists
__device__ __forceinline__ void ph_c_fill(const ContractArgs &A, int64_t t0, int64_t nt) {
    const Level &L = A.L;
    const Level &C = A.C;
    if (t0 == 0 && ipos_of(A, L.np) != newpos_of(A, L.np)) atomicOr(&A.box->err, E_INTERNAL);
    CSTRIDE_G(t, L.np, t0, nt) {
        if (!(A.kflag[t] & 1)) continue;
        const int32_t v = L.inode[t], c = A.gamma[v], u = A.rep_of[c];
        const int32_t other = v == u ? A.mate[u] : u;
        const int32_t x = L.inc[t];
        const int32_t va = L.ioff[v], vm = va + L.nin[v];
        const bool dst = t < (int64_t)vm;
        int32_t r = ipos_of(A, t) - ipos_of(A, dst ? va : vm);
        if (other >= 0) {
            const int32_t oa = L.ioff[other], om = oa + L.nin[other], ob = L.ioff[other + 1];
            const int32_t lo = dst ? oa : om, hi = dst ? om : ob;
            r += ipos_of(A, lower_bound_seg(L.inc, lo, hi, x)) - ipos_of(A, lo);
        }
        const int32_t pos = C.ioff[c] + (dst ? 0 : C.nin[c]) + r;
        if (pos < C.ioff[c + 1]) {
            C.inc[pos] = x;
            C.inode[pos] = c;
        } else {
            atomicOr(&A.box->err, E_INTERNAL);
        }
    }
}

__global__ void __cluster_dims__(SQ_CS, 1, 1) __launch_bounds__(SQ_T) k_contract_cluster(ContractArgs A) {
    HP_KERNEL_ENTER();
    __shared__ int32_t s_tmp[40];
    __shared__ int32_t s_part;
    __shared__ long long s_ll[40];
    __shared__ long long s_pll;
    cg::cluster_group cl = cg::this_cluster();
    if (contract_off(A.box)) return;   // uniform over the cluster
    const int64_t t0 = (int64_t)cl.block_rank() * blockDim.x + threadIdx.x, nt = (int64_t)SQ_CS * blockDim.x;
    const int32_t n = A.L.n, np = (int32_t)A.L.np;
    ph_c_flags(A, t0, nt);
    cl.sync();
    const int32_t cn = cluster_scan_excl<int32_t>(cl, A.isrep, A.cid, n, s_tmp, &s_part);
    const long long tot = cluster_scan_excl<long long>(cl, reinterpret_cast<long long *>(A.kflag),
                                                       reinterpret_cast<long long *>(A.kscan), np, s_ll, &s_pll);
    if (t0 == 0) {
        A.box->cn = cn;
        A.kscan[np] = tot;
    }
    cl.sync();
    ph_c_map(A, t0, nt);
    cl.sync();
    ph_c_pins(A, t0, nt);
    cl.sync();
    const int32_t total = cluster_scan_excl<int32_t>(cl, A.ccnt, A.C.ioff, n, s_tmp, &s_part);
    if (t0 == 0) A.C.ioff[n] = total;
    cl.sync();
    ph_c_fill(A, t0, nt);
}

__global__ void k_c_flags(ContractArgs A) {
    HP_KERNEL_ENTER();
    ph_c_flags(A, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}
__global__ void k_c_map(ContractArgs A) {
    HP_KERNEL_ENTER();
    if (contract_off(A.box)) return;
    ph_c_map(A, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}
__global__ void k_c_pins(ContractArgs A) {
    HP_KERNEL_ENTER();
    if (contract_off(A.box)) return;
    ph_c_pins(A, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}
__global__ void k_c_fill(ContractArgs A) {
    HP_KERNEL_ENTER();
    if (contract_off(A.box)) return;
    ph_c_fill(A, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

bool contract_level(const Level &L, const int32_t *mate, LevelBox *box, LevelBox *hb, Level &C, Arena &A) {
    cudaStream_t s = A.stream();
    const int32_t n = L.n, e = L.e;
    const int64_t np = L.np;
    ContractArgs X;
    X.L = L;
    X.mate = mate;
    X.box = box;
    X.isrep = A.get<int32_t>(n);
    X.cid = A.get<int32_t>(n);
    X.kflag = A.get<int64_t>(np);
    X.kscan = A.get<int64_t>(np + 1);
    X.rep_of = A.get<int32_t>(n);
    X.ccnt = A.get<int32_t>(n);
    // the coarse level at the fine level's sizes (nodes and pins only shrink)
    Level K;
    K.size = A.get<int32_t>(n);
    K.nbnd = A.get<int32_t>(n);
    K.off = A.get<int32_t>(e + 1);
    K.nsrc = A.get<int32_t>(e);
    K.pin = A.get<int32_t>(np);
    K.pedge = A.get<int32_t>(np);
    K.ioff = A.get<int32_t>(n + 1);
    K.nin = A.get<int32_t>(n);
    K.inc = A.get<int32_t>(np);
    K.inode = A.get<int32_t>(np);
    X.C = K;
    X.gamma = A.get<int32_t>(n);
    if (np <= CONTRACT_CLUSTER_NP && np > 0 && n > 0) {
        launch_k(k_contract_cluster, SQ_CS, SQ_T, 0, s, X);
        HP_LAUNCH_CHECK();
    } else {
        const int g = grid_of(std::max<int64_t>(n, np), 256);
        launch_k(k_c_flags, g, 256, 0, s, X);
        HP_LAUNCH_CHECK();
        scan_excl(X.isrep, X.cid, n, &box->cn, A);
        scan_excl(X.kflag, X.kscan, np, X.kscan + np, A);
        launch_k(k_c_map, grid_of(std::max<int64_t>(n, e), 256), 256, 0, s, X);
        HP_LAUNCH_CHECK();
        launch_k(k_c_pins, g, 256, 0, s, X);
        HP_LAUNCH_CHECK();
        scan_excl(X.ccnt, K.ioff, n, K.ioff + n, A);
        launch_k(k_c_fill, grid_of(np, 256), 256, 0, s, X);
        HP_LAUNCH_CHECK();
    }
    fetch_bytes(hb, box, sizeof(LevelBox), s);
    for (void *p : {(void *)X.isrep, (void *)X.cid, (void *)X.kflag, (void *)X.kscan, (void *)X.rep_of, (void *)X.ccnt})
        A.release(p);
    if (hb->pairs + hb->iso == 0) {
        for (void *p : {(void *)K.size, (void *)K.nbnd, (void *)K.off, (void *)K.nsrc, (void *)K.pin, (void *)K.pedge,
                        (void *)K.ioff, (void *)K.nin, (void *)K.inc, (void *)K.inode, (void *)X.gamma})
            A.release(p);
        return false;
    }
    const_cast<Level &>(L).gamma = X.gamma;
    C = K;
    C.n = hb->cn;
    C.e = e;
    C.np = hb->cnp;
    return true;
}

}  // namespace hp
