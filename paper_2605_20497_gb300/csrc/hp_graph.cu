// hp_graph.cu -- input checks, incidence sets (Sec. IV-B) and coarse
// hypergraph construction (Sec. V-E).
#include <cuda_runtime.h>

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
__global__ void k_rep_flags(const int32_t *mate, int32_t n, int32_t *isrep) {
    HP_KERNEL_ENTER();
    GRID_STRIDE(v, (int64_t)n) {
        int32_t m = mate[v];
        isrep[v] = (m < 0 || v < m) ? 1 : 0;
    }
}

__global__ void k_gamma(const int32_t *mate, const int32_t *cid, const int32_t *size, const int32_t *nbcnt, int32_t n,
                        int32_t *gamma, int32_t *csize, int32_t *cnb) {
    HP_KERNEL_ENTER();
    GRID_STRIDE(v, (int64_t)n) {
        int32_t m = mate[v];
        int32_t r = (m >= 0 && m < v) ? m : (int32_t)v;
        int32_t g = cid[r];
        gamma[v] = g;
        if (r == v) {
            csize[g] = size[v] + (m >= 0 ? size[m] : 0);
            int64_t b = (int64_t)nbcnt[v] + (m >= 0 ? nbcnt[m] : 0);
            cnb[g] = b > 0x7fffffff ? 0x7fffffff : (int32_t)b;
        }
    }
}

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
__global__ void k_keep(const int32_t *pin, const int32_t *pedge, const int32_t *off, const int32_t *nsrc,
                       const int32_t *mate, const int32_t *ioff, const int32_t *inc, const int32_t *nin, int64_t np,
                       int32_t *keep) {
    HP_KERNEL_ENTER();
    GRID_STRIDE(j, np) {
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
        keep[j] = k;
    }
}

__global__ void k_coarse_edges(const int32_t *off, const int32_t *nsrc, const int32_t *newpos, int32_t e,
                               int32_t *coff, int32_t *cnsrc) {
    HP_KERNEL_ENTER();
    GRID_STRIDE(i, (int64_t)e) {
        int32_t a = newpos[off[i]];
        coff[i] = a;
        cnsrc[i] = newpos[off[i] + nsrc[i]] - a;
    }
}

__global__ void k_coarse_pins(const int32_t *pin, const int32_t *pedge, const int32_t *keep, const int32_t *newpos,
                              const int32_t *gamma, int64_t np, int32_t *cpin, int32_t *cpedge) {
    HP_KERNEL_ENTER();
    GRID_STRIDE(j, np) {
        if (keep[j]) {
            int32_t k = newpos[j];
            cpin[k] = gamma[pin[j]];
            cpedge[k] = pedge[j];
        }
    }
}

bool contract_level(const Level &L, const int32_t *mate, LevelBox *box, LevelBox *hb, Level &C, Arena &A) {
    cudaStream_t s = A.stream();
    int32_t *isrep = A.get<int32_t>(L.n);
    int32_t *cid = A.get<int32_t>(L.n + 1);
    launch_k(k_rep_flags, grid_of(L.n, 256), 256, 0, s, mate, L.n, isrep);
    HP_LAUNCH_CHECK();
    scan_excl(isrep, cid, L.n, &box->cn, A);
    int32_t *keep = A.get<int32_t>(L.np);
    int32_t *newpos = A.get<int32_t>(L.np + 1);
    if (L.np) {
        launch_k(k_keep, grid_of(L.np, 256), 256, 0, s, L.pin, L.pedge, L.off, L.nsrc, mate, L.ioff, L.inc, L.nin, L.np,
                                                   keep);
        HP_LAUNCH_CHECK();
    }
    scan_excl(keep, newpos, L.np, &box->cnp, A);
    HPC(cudaMemcpyAsync(newpos + L.np, &box->cnp, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    fetch_bytes(hb, box, sizeof(LevelBox), s);
    if (hb->pairs + hb->iso == 0) {
        for (void *p : {(void *)isrep, (void *)cid, (void *)keep, (void *)newpos}) A.release(p);
        return false;
    }
    C.n = hb->cn;
    C.e = L.e;
    C.np = hb->cnp;
    C.size = A.get<int32_t>(C.n);
    C.nbnd = A.get<int32_t>(C.n);
    const_cast<Level &>(L).gamma = A.get<int32_t>(L.n);
    launch_k(k_gamma, grid_of(L.n, 256), 256, 0, s, mate, cid, L.size, L.nbnd, L.n, L.gamma, C.size, C.nbnd);
    HP_LAUNCH_CHECK();
    A.release(isrep);
    A.release(cid);
    C.off = A.get<int32_t>(C.e + 1);
    C.nsrc = A.get<int32_t>(C.e);
    C.pin = A.get<int32_t>(C.np);
    C.pedge = A.get<int32_t>(C.np);
    if (C.e > 0) {
        launch_k(k_coarse_edges, grid_of(C.e, 256), 256, 0, s, L.off, L.nsrc, newpos, C.e, C.off, C.nsrc);
        HP_LAUNCH_CHECK();
    }
    HPC(cudaMemcpyAsync(C.off + C.e, newpos + L.np, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    if (L.np) {
        launch_k(k_coarse_pins, grid_of(L.np, 256), 256, 0, s, L.pin, L.pedge, keep, newpos, L.gamma, L.np, C.pin, C.pedge);
        HP_LAUNCH_CHECK();
    }
    A.release(keep);
    A.release(newpos);
    build_incidence(C, A);
    return true;
}

}  // namespace hp
