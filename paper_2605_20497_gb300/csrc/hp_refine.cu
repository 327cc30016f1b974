// hp_refine.cu -- one level of refinement (Sec. VI): Theta repetitions of
//   pins(p,e) lists  -> move proposal by gain (Eq. 13, Sec. VI-B)
//   -> sort (p_s asc, gain desc, node asc) -> chaining (Sec. VI-C)
//   -> chain order -> in-sequence gains (Eq. 14-15, exact change of
//   connectivity) -> event-based validity of every prefix (Sec. VI-D)
//   -> apply the best valid prefix.
// pins(p,e) is kept as a short list per hyperedge, sorted by partition id, at
// the hyperedge's own pin segment: (p, pins(p,e), pins_in(p,e)).
#include <cuda_runtime.h>

#include <cstring>

#include <algorithm>
#include <climits>
#include <initializer_list>

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

struct Plist {
    int32_t *p = nullptr, *cnt = nullptr, *cin = nullptr;  // [np]
    int32_t *lam = nullptr;                                // [e] entries per hyperedge
};

// slot of key x in a table of mask + 1 (a power of two, >= 2) slots: the top
// bits of a Fibonacci product, so that keys with equal low bits spread out
__device__ __forceinline__ uint32_t hslot(int32_t x, uint32_t mask) {
    return mask ? ((uint32_t)x * 0x9E3779B1u) >> __clz(mask) : 0u;
}

template <int G> __device__ __forceinline__ void gsync() {
    if (G == 32) __syncwarp();
    else __syncthreads();
}

// ---------------------------------------------------------------- pins(p,e)
// One group of G threads builds the sorted list of hyperedge e.  Its table
// of `cap` slots (keys/cnt/cin) is clean (keys -1, counters 0) on entry and
// is left clean; the entry buffers hold >= |e| slots.  Both live in shared
// or global memory private to the group.  Optionally adds D(p) (distinct
// inbound hyperedges per part) and saving(v) for the hyperedge's pins (v
// alone in its part, |e| >= 2).
template <int G>
__device__ void plist_edge(int32_t e, int gt, const int32_t *off, const int32_t *pin, const int32_t *nsrc,
                           const int32_t *w, const int32_t *rho, int32_t *keys, int32_t *tc, int32_t *tci, uint32_t cap,
                           int32_t *ent_s, int32_t *ent_p, int32_t *ent_c, int32_t *ent_ci, int32_t *g_cnt, Plist PL,
                           int32_t *D, long long *saving) {
    const uint32_t mask = cap - 1;
    const int32_t a = off[e], b = off[e + 1], dst0 = a + nsrc[e];
    if (gt == 0) *g_cnt = 0;
    gsync<G>();
    for (int32_t j = a + gt; j < b; j += G) {
        int32_t p = rho[pin[j]];
        uint32_t h = hslot(p, mask);
        for (uint32_t probe = 0; probe < cap; probe++) {
            int32_t k = ((volatile int32_t *)keys)[h];
            if (k == -1) {
                int32_t old = atomicCAS(&keys[h], -1, p);
                if (old == -1) {
                    ent_s[atomicAdd(g_cnt, 1)] = (int32_t)h;
                    k = p;
                } else {
                    k = old;
                }
            }
            if (k == p) {
                atomicAdd(&tc[h], 1);
                if (j >= dst0) atomicAdd(&tci[h], 1);
                break;
            }
            h = (h + 1) & mask;
        }
    }
    gsync<G>();
    const int32_t lam = *(volatile int32_t *)g_cnt;
    if (saving && b - a >= 2) {
        const long long we = w[e];
        for (int32_t j = a + gt; j < b; j += G) {
            int32_t v = pin[j], p = rho[v];
            uint32_t h = hslot(p, mask);
            for (uint32_t probe = 0; probe < cap && keys[h] != p; probe++) h = (h + 1) & mask;
            if (keys[h] == p && tc[h] == 1) atomicAdd((unsigned long long *)&saving[v], (unsigned long long)we);
        }
    }
    for (int32_t i = gt; i < lam; i += G) {
        int32_t h = ent_s[i];
        ent_p[i] = keys[h];
        ent_c[i] = tc[h];
        ent_ci[i] = tci[h];
    }
    gsync<G>();
    for (int32_t i = gt; i < lam; i += G) {
        int32_t p = ent_p[i], r = 0;
        for (int32_t k = 0; k < lam; k++) r += ent_p[k] < p;
        PL.p[a + r] = p;
        PL.cnt[a + r] = ent_c[i];
        PL.cin[a + r] = ent_ci[i];
        if (D && ent_ci[i] > 0) atomicAdd(&D[p], 1);
        int32_t h = ent_s[i];
        keys[h] = -1;
        tc[h] = 0;
        tci[h] = 0;
    }
    if (gt == 0) PL.lam[e] = lam;
    gsync<G>();
}

constexpr int PLW_T = 128;  // warp-per-edge kernel: 4 warps
constexpr int32_t MID_SPLIT = 128;   // warp-tier hyperedges up to this size get small tables

// edges with |e| <= small_max, one warp each, tables in shared memory
__global__ void __launch_bounds__(PLW_T) k_plist_small(const int32_t *off, const int32_t *pin, const int32_t *nsrc,
                                                       const int32_t *w, const int32_t *rho, int32_t e,
                                                       const int32_t *list, int32_t small_max, uint32_t cap, Plist PL,
                                                       int32_t *D, long long *saving, int32_t skip_below,
                                                       int32_t skip_above) {
    HP_KERNEL_ENTER();
    extern __shared__ __align__(16) int32_t sm[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // table of cap slots; entry buffers of cap / 2 >= lambda(e) entries
    const int per = 5 * (int)cap + 1, ent = (int)cap / 2;
    int32_t *base = sm + wid * per;
    int32_t *keys = base, *tc = base + cap, *tci = base + 2 * cap;
    int32_t *es = base + 3 * cap, *ep = es + ent, *ec = ep + ent, *eci = ec + ent, *gcnt = eci + ent;
    for (uint32_t i = lane; i < cap; i += 32) {
        keys[i] = -1;
        tc[i] = 0;
        tci[i] = 0;
    }
    __syncwarp();
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // all hyperedges up to small_max pins, or the given list (count e) skipping
    // the ones of at most skip_below or more than skip_above pins
    for (int64_t i = warp; i < e; i += nw) {
        const int32_t ed = list ? list[i] : (int32_t)i;
        const int32_t sz = off[ed + 1] - off[ed];
        if ((!list && sz > small_max) || sz <= skip_below || sz > skip_above) continue;
        plist_edge<32>(ed, lane, off, pin, nsrc, w, rho, keys, tc, tci, cap, es, ep, ec, eci, gcnt, PL, D, saving);
    }
}

// edges with |e| > small_max, one CTA each, tables in global memory
__global__ void __launch_bounds__(256) k_plist_big(const int32_t *off, const int32_t *pin, const int32_t *nsrc,
                                                   const int32_t *w, const int32_t *rho, const int32_t *list,
                                                   int32_t count, uint32_t cap, int32_t *gtab, int32_t max_e, Plist PL,
                                                   int32_t *D, long long *saving) {
    HP_KERNEL_ENTER();
    __shared__ int32_t gcnt;
    int32_t *mine = gtab + (int64_t)blockIdx.x * (3 * (int64_t)cap + 4 * (int64_t)max_e);
    int32_t *keys = mine, *tc = mine + cap, *tci = mine + 2 * cap;
    int32_t *es = mine + 3 * cap, *ep = es + max_e, *ec = ep + max_e, *eci = ec + max_e;
    for (uint32_t i = threadIdx.x; i < cap; i += 256) {
        keys[i] = -1;
        tc[i] = 0;
        tci[i] = 0;
    }
    __syncthreads();
    for (int32_t k = blockIdx.x; k < count; k += gridDim.x)
        plist_edge<256>(list[k], threadIdx.x, off, pin, nsrc, w, rho, keys, tc, tci, cap, es, ep, ec, eci, &gcnt, PL,
                        D, saving);
}

__global__ void k_big_edges(const int32_t *off, int32_t e, int32_t small_max, int32_t *list, int32_t *cnt,
                            int32_t *maxe) {
    HP_KERNEL_ENTER();
    GRID_STRIDE(i, (int64_t)e) {
        int32_t sz = off[i + 1] - off[i];
        if (sz > small_max) {
            list[atomicAdd(cnt, 1)] = (int32_t)i;
            atomicMax(maxe, sz);
        }
    }
}

__global__ void k_max_edge(const int32_t *off, int32_t e, int32_t *maxe) {
    HP_KERNEL_ENTER();
    int32_t m = 0;
    GRID_STRIDE(i, (int64_t)e) m = max(m, off[i + 1] - off[i]);
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(maxe, m);
}

static uint32_t pow2_at_least(int64_t x) {
    uint32_t c = 1;
    while ((int64_t)c < x) c <<= 1;
    return c;
}

static void build_plist(const Level &L, const int32_t *w, const int32_t *rho, int32_t max_e, Plist &PL, int32_t *D,
                        long long *saving, Arena &A) {
    cudaStream_t s = A.stream();
    if (L.e == 0) return;
    const int32_t small_max = std::min<int32_t>(std::max<int32_t>(max_e, 1), 512);
    const uint32_t cap = pow2_at_least(2 * (int64_t)small_max);
    const int per = 5 * (int)cap + 1;
    size_t sm = (size_t)per * 4 * (PLW_T / 32);
    int occ = prepare_kernel((const void *)k_plist_small, PLW_T, sm);
    int grid = (int)std::min<int64_t>(cdiv(L.e, PLW_T / 32), (int64_t)num_sms() * std::max(occ, 1));
    launch_k(k_plist_small, std::max(grid, 1), PLW_T, sm, s, L.off, L.pin, L.nsrc, w, rho, L.e, nullptr, small_max, cap,
             PL, D, saving, 0, INT32_MAX);
    HP_LAUNCH_CHECK();
    if (max_e > small_max) {
        int32_t *list = A.get<int32_t>(L.e);
        int32_t *cnt = A.get<int32_t>(2);
        HPC(cudaMemsetAsync(cnt, 0, 2 * sizeof(int32_t), s));
        launch_k(k_big_edges, grid_of(L.e, 256), 256, 0, s, L.off, L.e, small_max, list, cnt, cnt + 1);
        HP_LAUNCH_CHECK();
        int32_t hc[2];
        fetch_bytes(hc, cnt, sizeof hc, s);
        if (hc[0] > 0) {
            uint32_t bcap = pow2_at_least(2 * (int64_t)hc[1]);
            int nb = std::min<int>(hc[0], num_sms() * 2);
            int32_t *gtab = A.get<int32_t>((int64_t)nb * (3 * (int64_t)bcap + 4 * (int64_t)hc[1]));
            launch_k(k_plist_big, nb, 256, 0, s, L.off, L.pin, L.nsrc, w, rho, list, hc[0], bcap, gtab, hc[1], PL, D,
                     saving);
            HP_LAUNCH_CHECK();
            A.release(gtab);
        }
        A.release(list);
        A.release(cnt);
    }
}

// ---------------------------------------------------------------- objective
__global__ void k_objective(const int32_t *lam, const int32_t *w, int32_t e, unsigned long long *conn,
                            unsigned long long *cutnet) {
    HP_KERNEL_ENTER();
    unsigned long long c = 0, cn = 0;
    GRID_STRIDE(i, (int64_t)e) {
        int32_t l = lam[i];
        c += (unsigned long long)w[i] * (unsigned long long)(l - 1);
        if (l > 1) cn += (unsigned long long)w[i];
    }
    for (int o = 16; o > 0; o >>= 1) {
        c += __shfl_down_sync(0xffffffffu, c, o);
        cn += __shfl_down_sync(0xffffffffu, cn, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(conn, c);
        atomicAdd(cutnet, cn);
    }
}

void objective(const Level &L, const int32_t *w, const int32_t *rho, int32_t nparts, int64_t *conn_dev,
               int64_t *cutnet_dev, Arena &A) {
    cudaStream_t s = A.stream();
    (void)nparts;
    HPC(cudaMemsetAsync(conn_dev, 0, sizeof(int64_t), s));
    HPC(cudaMemsetAsync(cutnet_dev, 0, sizeof(int64_t), s));
    if (L.e == 0) return;
    int32_t *maxe = A.get<int32_t>(1);
    HPC(cudaMemsetAsync(maxe, 0, sizeof(int32_t), s));
    launch_k(k_max_edge, grid_of(L.e, 256), 256, 0, s, L.off, L.e, maxe);
    HP_LAUNCH_CHECK();
    int32_t me = fetch<int32_t>(maxe, s);
    Plist PL;
    PL.p = A.get<int32_t>(L.np);
    PL.cnt = A.get<int32_t>(L.np);
    PL.cin = A.get<int32_t>(L.np);
    PL.lam = A.get<int32_t>(L.e);
    build_plist(L, w, rho, me, PL, nullptr, nullptr, A);
    launch_k(k_objective, grid_of(L.e, 256), 256, 0, s, PL.lam, w, L.e, (unsigned long long *)conn_dev,
             (unsigned long long *)cutnet_dev);
    HP_LAUNCH_CHECK();
    A.release(PL.p);
    A.release(PL.cnt);
    A.release(PL.cin);
    A.release(PL.lam);
    A.release(maxe);
}

// ---------------------------------------------------------------- Eq. 13 gains
struct Moves {
    int32_t *node, *src, *dst;
    long long *gain;
    int32_t *count;
};

constexpr int GN_T = 128;

// gain(v,p) = saving(v) - loss(v,p) with loss = W(v) - conn(v,p), conn(v,p) =
// sum of w(e) over e in I(v) with pins(p,e) > 0 (singleton hyperedges cancel).
__device__ void gains_node(int32_t v, const int32_t *off, const int32_t *ioff, const int32_t *inc, const int32_t *w,
                           const int32_t *rho, const int32_t *size, const long long *psize, const long long *saving,
                           const long long *wns, Plist PL, int32_t omega, int second_half, int32_t *keys,
                           long long *conn, int32_t *slots, uint32_t cap, uint32_t limit, int32_t *s_cnt, int *s_flag,
                           Moves M,
                           int32_t *ovf, int32_t *ovf_n, long long *s_rg, int32_t *s_rp) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t mask = cap - 1;
    const int32_t s = rho[v];
    auto add = [&](int32_t p, long long we) {
        uint32_t h = hslot(p, mask);
        for (uint32_t probe = 0; probe < cap; probe++) {
            int32_t kk = ((volatile int32_t *)keys)[h];
            if (kk == -1) {
                int32_t old = atomicCAS(&keys[h], -1, p);
                if (old == -1) {
                    const uint32_t slot = (uint32_t)atomicAdd(s_cnt, 1);
                    if (slot < limit) slots[slot] = (int32_t)h;
                    else *(volatile int *)s_flag = 1;
                    kk = p;
                } else {
                    kk = old;
                }
            }
            if (kk == p) {
                atomicAdd((unsigned long long *)&conn[h], (unsigned long long)we);
                return;
            }
            h = (h + 1) & mask;
        }
    };
    // one cut hyperedge per thread.  The k-th entries of the pins lists of a
    // warp's 32 hyperedges are combined by part across the warp (match_any)
    // before one table update per distinct part, so that the few parts a
    // node touches are not hammered by every lane.
    {
        const int32_t c0 = ioff[v], c1 = ioff[v + 1];
        for (int32_t base = c0; base < c1; base += blockDim.x) {
            if (__any_sync(0xffffffffu, *(volatile int *)s_flag)) break;
            const int32_t t = base + (int32_t)threadIdx.x;
            int32_t a = 0, lam = 0;
            uint32_t we = 0;
            if (t < c1) {
                const int32_t e = inc[t];
                lam = PL.lam[e];
                a = off[e];
                we = (uint32_t)w[e];
            }
            const int kmax = __reduce_max_sync(0xffffffffu, (unsigned)lam);
            for (int k = 0; k < kmax; k++) {
                int32_t p = k < lam ? PL.p[a + k] : -1;
                if (p == s) p = -1;
                const unsigned m = __match_any_sync(0xffffffffu, p);
                const unsigned sw = __reduce_add_sync(m, p >= 0 ? we : 0u);
                if (p >= 0 && lane == __ffs(m) - 1) add(p, (long long)sw);
            }
        }
    }
    __syncthreads();
    const int overflow = *s_flag;
    long long bg = 0;
    int32_t bp = -1;
    const long long base = saving[v] - wns[v];
    if (overflow) {
        // the slot list is incomplete: clear the whole table, redo the node in a larger one
        for (uint32_t h = threadIdx.x; h < cap; h += blockDim.x) {
            keys[h] = -1;
            conn[h] = 0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            ovf[atomicAdd(ovf_n, 1)] = v;
            *s_flag = 0;
            *s_cnt = 0;
        }
        __syncthreads();
        return;
    }
    const int32_t used = *(volatile int32_t *)s_cnt;
    for (int32_t i = threadIdx.x; i < used; i += blockDim.x) {
        const int32_t h = slots[i];
        const int32_t p = keys[h];
        if (!second_half || (long long)size[v] + psize[p] <= omega) {
            long long g = base + conn[h];
            if (bp < 0 || g > bg || (g == bg && p > bp)) {
                bg = g;
                bp = p;
            }
        }
        keys[h] = -1;
        conn[h] = 0;
    }
    for (int o = 16; o > 0; o >>= 1) {
        long long og = __shfl_down_sync(0xffffffffu, bg, o);
        int32_t op = __shfl_down_sync(0xffffffffu, bp, o);
        if (op >= 0 && (bp < 0 || og > bg || (og == bg && op > bp))) {
            bg = og;
            bp = op;
        }
    }
    if (lane == 0) {
        s_rg[wid] = bg;
        s_rp[wid] = bp;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < nw; k++) {
            if (s_rp[k] >= 0 && (bp < 0 || s_rg[k] > bg || (s_rg[k] == bg && s_rp[k] > bp))) {
                bg = s_rg[k];
                bp = s_rp[k];
            }
        }
        if (bp >= 0 && bg > 0) {
            int32_t i = atomicAdd(M.count, 1);
            M.node[i] = v;
            M.src[i] = s;
            M.dst[i] = bp;
            M.gain[i] = bg;
        }
        *s_cnt = 0;
    }
    __syncthreads();
}

struct GainArgs {
    const int32_t *off, *ioff, *inc, *w, *rho, *size;
    const long long *psize, *saving, *wns;
    Plist PL;
    int32_t omega;
    int second_half;
    Moves M;
};

template <int BT>
__global__ void __launch_bounds__(BT) k_gains_smem(GainArgs G, const int32_t *list, const int32_t *count_p,
                                                     uint32_t cap, int32_t *ovf, int32_t *ovf_n) {
    HP_KERNEL_ENTER();
    const int32_t count = *count_p;
    extern __shared__ __align__(16) unsigned char smem[];
    long long *conn = reinterpret_cast<long long *>(smem);
    int32_t *keys = reinterpret_cast<int32_t *>(conn + cap);
    int32_t *slots = keys + cap;
    __shared__ int32_t s_cnt;
    __shared__ int s_flag;
    __shared__ long long s_rg[32];
    __shared__ int32_t s_rp[32];
    for (uint32_t i = threadIdx.x; i < cap; i += BT) {
        keys[i] = -1;
        conn[i] = 0;
    }
    if (threadIdx.x == 0) {
        s_cnt = 0;
        s_flag = 0;
    }
    __syncthreads();
    for (int32_t k = blockIdx.x; k < count; k += gridDim.x)
        gains_node(list[k], G.off, G.ioff, G.inc, G.w, G.rho, G.size, G.psize, G.saving, G.wns, G.PL, G.omega,
                   G.second_half, keys, conn, slots, cap, cap * 3 / 4, &s_cnt, &s_flag, G.M, ovf, ovf_n, s_rg, s_rp);
}

__global__ void __launch_bounds__(GN_T) k_gains_global(GainArgs G, const int32_t *list, const int32_t *count_p,
                                                       uint32_t cap, int32_t *gkeys, long long *gconn, int32_t *bad,
                                                       int32_t *bad_n) {
    HP_KERNEL_ENTER();
    const int32_t count = *count_p;
    if (count == 0) return;
    __shared__ int32_t s_cnt;
    __shared__ int s_flag;
    __shared__ long long s_rg[8];
    __shared__ int32_t s_rp[8];
    int32_t *keys = gkeys + (int64_t)blockIdx.x * 2 * cap;
    int32_t *slots = keys + cap;
    long long *conn = gconn + (int64_t)blockIdx.x * cap;
    for (uint32_t i = threadIdx.x; i < cap; i += GN_T) {
        keys[i] = -1;
        conn[i] = 0;
    }
    if (threadIdx.x == 0) {
        s_cnt = 0;
        s_flag = 0;
    }
    __syncthreads();
    for (int32_t k = blockIdx.x; k < count; k += gridDim.x)
        gains_node(list[k], G.off, G.ioff, G.inc, G.w, G.rho, G.size, G.psize, G.saving, G.wns, G.PL, G.omega,
                   G.second_half, keys, conn, slots, cap, cap - 1, &s_cnt, &s_flag, G.M, bad, bad_n, s_rg, s_rp);
}

// Nodes with at most GW_DEG cut hyperedges: one warp each, with a warp-private
// table of GW_SLOTS parts in shared memory.  Entries of the lanes' hyperedges
// are combined by part across the warp before each table update.  A node
// whose neighbouring parts outgrow `limit` is handed to the CTA kernel's list.
constexpr int GW_T = 256, GW_SLOTS = 256;
__global__ void __launch_bounds__(GW_T) k_gains_warp(GainArgs G, const int32_t *list, const int32_t *count_p,
                                                     uint32_t limit, int32_t *spill, int32_t *spill_n) {
    HP_KERNEL_ENTER();
    __shared__ int32_t s_keys[GW_T / 32][GW_SLOTS];
    __shared__ long long s_conn[GW_T / 32][GW_SLOTS];
    __shared__ int32_t s_used[GW_T / 32];
    const unsigned FULL = 0xffffffffu;
    const int32_t count = *count_p;
    if (count == 0) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t *keys = s_keys[wid];
    long long *conn = s_conn[wid];
    for (int h = lane; h < GW_SLOTS; h += 32) {
        keys[h] = -1;
        conn[h] = 0;
    }
    if (lane == 0) s_used[wid] = 0;
    __syncwarp();
    const int64_t gw = (int64_t)blockIdx.x * (GW_T / 32) + wid, nw = (int64_t)gridDim.x * (GW_T / 32);
    for (int64_t k = gw; k < count; k += nw) {
        const int32_t v = list[k];
        const int32_t s = G.rho[v];
        const int32_t c0 = G.ioff[v], c1 = G.ioff[v + 1];
        for (int32_t base = c0; base < c1; base += 32) {
            if (*(volatile int32_t *)&s_used[wid] > (int32_t)limit) break;   // same value for the whole warp
            const int32_t t = base + lane;
            int32_t a = 0, lam = 0;
            uint32_t we = 0;
            if (t < c1) {
                const int32_t e = G.inc[t];
                lam = G.PL.lam[e];
                a = G.off[e];
                we = (uint32_t)G.w[e];
            }
            const int kmax = (int)__reduce_max_sync(FULL, (unsigned)lam);
            for (int k2 = 0; k2 < kmax; k2++) {
                int32_t p = k2 < lam ? G.PL.p[a + k2] : -1;
                if (p == s) p = -1;
                const unsigned m = __match_any_sync(FULL, p);
                const unsigned sw = __reduce_add_sync(m, p >= 0 ? we : 0u);
                if (p >= 0 && lane == __ffs(m) - 1) {
                    uint32_t h = hslot(p, GW_SLOTS - 1);
                    for (int probe = 0; probe < GW_SLOTS; probe++) {
                        int32_t kk = ((volatile int32_t *)keys)[h];
                        if (kk == -1) {
                            const int32_t old = atomicCAS(&keys[h], -1, p);
                            if (old == -1) {
                                atomicAdd(&s_used[wid], 1);
                                kk = p;
                            } else {
                                kk = old;
                            }
                        }
                        if (kk == p) {
                            atomicAdd((unsigned long long *)&conn[h], (unsigned long long)sw);
                            break;
                        }
                        h = (h + 1) & (GW_SLOTS - 1);
                    }
                }
            }
            __syncwarp();
        }
        __syncwarp();
        const bool spilled = *(volatile int32_t *)&s_used[wid] > (int32_t)limit;
        const long long basev = G.saving[v] - G.wns[v];
        long long bg = 0;
        int32_t bp = -1;
        for (int h = lane; h < GW_SLOTS; h += 32) {
            const int32_t p = keys[h];
            if (p >= 0 && !spilled && (!G.second_half || (long long)G.size[v] + G.psize[p] <= G.omega)) {
                const long long g = basev + conn[h];
                if (bp < 0 || g > bg || (g == bg && p > bp)) {
                    bg = g;
                    bp = p;
                }
            }
            keys[h] = -1;
            conn[h] = 0;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const long long og = __shfl_down_sync(FULL, bg, o);
            const int32_t op = __shfl_down_sync(FULL, bp, o);
            if (op >= 0 && (bp < 0 || og > bg || (og == bg && op > bp))) {
                bg = og;
                bp = op;
            }
        }
        if (lane == 0) {
            if (spilled) {
                spill[atomicAdd(spill_n, 1)] = v;
            } else if (bp >= 0 && bg > 0) {
                const int32_t i = atomicAdd(G.M.count, 1);
                G.M.node[i] = v;
                G.M.src[i] = s;
                G.M.dst[i] = bp;
                G.M.gain[i] = bg;
            }
            s_used[wid] = 0;
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------- per level constants
// Per node: Wns(v) = sum of w(e) over incident hyperedges with |e| >= 2, and
// the number of singleton hyperedges {v} that hold v as a destination.
// Singleton hyperedges cancel in every gain (they are spared and re-created
// by any move) and change only the distinct-inbound count, by one per
// singleton at p_s (-) and at p_d (+): they are handled per node.
__global__ void k_level_nodes(const int32_t *off, const int32_t *ioff, const int32_t *inc, const int32_t *inode,
                              const int32_t *nin, const int32_t *w, int64_t np, long long *wns, int32_t *singin) {
    HP_KERNEL_ENTER();
    const int lane = threadIdx.x & 31;
    const int64_t wbase = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) << 5;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = wbase; base < np; base += stride) {
        const int64_t t = base + lane;
        const bool valid = t < np;
        const int32_t v = valid ? inode[t] : -1 - lane;
        long long a = 0;
        int32_t c = 0;
        if (valid) {
            const int32_t e = inc[t];
            const int32_t sz = off[e + 1] - off[e];
            if (sz >= 2) a = w[e];
            else if (t < ioff[v] + nin[v]) c = 1;
        }
        bool tail = warp_run_sum(v, a);
        warp_run_sum(v, c);
        if (valid && tail) {
            if (a) atomicAdd((unsigned long long *)&wns[v], (unsigned long long)a);
            if (c) atomicAdd(&singin[v], c);
        }
    }
}

// hyperedges with >= 2 pins: up to TINY_E pins (one thread each), up to
// small_max (a warp each), larger (a CTA each).  All of them form `act`
// (the in-sequence pass); tiny ones are also listed apart.
constexpr int TINY_E = 8;
// largest hyperedge handled a warp each: the level's largest, at least 2, at most 512
__host__ __device__ inline int32_t level_small_max(int32_t max_e) { return max_e < 2 ? 2 : (max_e > 512 ? 512 : max_e); }
__global__ void k_level_edges(const int32_t *off, int32_t e, const int32_t *max_e, int32_t *act, int32_t *big,
                              int32_t *tiny, int32_t *mid, int32_t *cnt) {
    HP_KERNEL_ENTER();
    const int32_t small_max = level_small_max(*max_e);
    GRID_STRIDE(i, (int64_t)e) {
        int32_t sz = off[i + 1] - off[i];
        if (sz >= 2 && sz <= small_max) {
            act[atomicAdd(&cnt[0], 1)] = (int32_t)i;
            if (sz <= TINY_E) tiny[atomicAdd(&cnt[3], 1)] = (int32_t)i;
            else mid[atomicAdd(&cnt[4], 1)] = (int32_t)i;
        } else if (sz > small_max) big[atomicAdd(&cnt[1], 1)] = (int32_t)i;
    }
}

// pins(p, e) list of a hyperedge of 2..TINY_E pins by one thread.  D(p) and
// saving(v) updates are combined across the warp by key (match_any) first:
// a coarse node or a part shared by many neighbouring hyperedges would
// otherwise take one global atomic per hyperedge.
__global__ void k_plist_tiny(const int32_t *off, const int32_t *pin, const int32_t *nsrc, const int32_t *w,
                             const int32_t *rho, const int32_t *list, int32_t count, Plist PL, int32_t *D,
                             long long *saving) {
    HP_KERNEL_ENTER();
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < count; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = base + threadIdx.x;
        const bool live = k < count;
        int32_t a = 0, sz = 0, dst0 = 0;
        uint32_t we = 0;
        if (live) {
            const int32_t e = list[k];
            a = off[e];
            sz = off[e + 1] - a;
            dst0 = nsrc[e];
            we = (uint32_t)w[e];
        }
        int32_t vv[TINY_E], pp[TINY_E], up[TINY_E], uc[TINY_E], uci[TINY_E];
        int32_t nu = 0;
#pragma unroll
        for (int j = 0; j < TINY_E; j++) {
            vv[j] = -1;
            pp[j] = -1;
            up[j] = 0x7fffffff;
            uc[j] = 0;
            uci[j] = 0;
        }
#pragma unroll
        for (int j = 0; j < TINY_E; j++) {
            if (j < sz) {
                vv[j] = pin[a + j];
                pp[j] = rho[vv[j]];
            }
        }
#pragma unroll
        for (int j = 0; j < TINY_E; j++) {
            if (j >= sz) break;
            const int32_t p = pp[j];
            int32_t f = -1;
#pragma unroll
            for (int u = 0; u < TINY_E; u++)
                if (u < nu && up[u] == p) f = u;
            if (f < 0) f = nu++;
#pragma unroll
            for (int u = 0; u < TINY_E; u++)
                if (u == f) {
                    up[u] = p;
                    uc[u]++;
                    uci[u] += j >= dst0;
                }
        }
        // sorted by part id: rank of each distinct entry
#pragma unroll
        for (int u = 0; u < TINY_E; u++) {
            if (u < nu) {
                int32_t r = 0;
#pragma unroll
                for (int x = 0; x < TINY_E; x++)
                    if (x < nu && up[x] < up[u]) r++;
                PL.p[a + r] = up[u];
                PL.cnt[a + r] = uc[u];
                PL.cin[a + r] = uci[u];
            }
        }
        if (live) PL.lam[list[k]] = nu;
        if (D) {
#pragma unroll
            for (int u = 0; u < TINY_E; u++) {
                const int32_t key = (u < nu && uci[u] > 0) ? up[u] : -1;
                const unsigned m = __match_any_sync(FULL, key);
                if (key >= 0 && lane == __ffs(m) - 1) atomicAdd(&D[key], __popc(m));
            }
        }
        if (saving) {
#pragma unroll
            for (int j = 0; j < TINY_E; j++) {
                int32_t c = 0;
#pragma unroll
                for (int u = 0; u < TINY_E; u++)
                    if (u < nu && up[u] == pp[j]) c = uc[u];
                const int32_t key = (j < sz && c == 1) ? vv[j] : -1;
                const unsigned m = __match_any_sync(FULL, key);
                const unsigned sw = __reduce_add_sync(m, key >= 0 ? we : 0u);
                if (key >= 0 && lane == __ffs(m) - 1)
                    atomicAdd((unsigned long long *)&saving[key], (unsigned long long)sw);
            }
        }
    }
}

// counters of one repetition (device)
enum { C_CAND, C_MOVES, C_OVF, C_BAD, C_NH, C_BAD0, C_APPLIED, C_NV, C_HUB, C_CW, C_TOUCH, C_TTOUCH,
       C_ACC,          // three 64-bit byte counters (even index: 8-byte aligned), see k_cut_flags
       C_N = C_ACC + 6 };

// moves of at most SMALLM are validated by one CTA (k_val_small) with the
// sorts in shared memory; moves of at most sq_max<uint64_t>() are sequenced by one
// thread-block cluster (k_seq_cluster); more take the multi-kernel path
constexpr int SMALLM = 6144, SEQ_T = 1024;
// refinement levels of at most this many nodes run their repetitions on the
// cluster kernels with one read-back each (every move count fits them)
constexpr int32_t SMALL_LEVEL = 32768;

#define STRIDE(i, n, t0, nt) for (int64_t i = (t0); i < (int64_t)(n); i += (nt))
#define G_T0 (blockIdx.x * (int64_t)blockDim.x + threadIdx.x)
#define G_NT ((int64_t)gridDim.x * blockDim.x)

struct RepArrays {
    int32_t n, e, nparts, rounds;
    int32_t *cnt, *linked;
    int32_t *D0;
    long long *psize, *saving;
    int32_t *pc;
    int32_t *pred, *succ, *chain, *mvpos;
    long long *cgain;
    unsigned long long *gseq, *acc0;
    int32_t *dDs, *dDd, *viol;
};

__device__ __forceinline__ int64_t rep_zero_span(const RepArrays &R) {
    return max(max((int64_t)R.n, (int64_t)R.nparts + 1), max((int64_t)C_N, (int64_t)R.rounds + 1));
}
// keep: the partition is the one of the previous repetition (it applied
// nothing), so D(p), |p| and saving(v) are still valid
__global__ void k_rep_zero(RepArrays R, int keep) {
    HP_KERNEL_ENTER();
    GRID_STRIDE(i, rep_zero_span(R)) {
        if (i < R.nparts && !keep) {
            R.D0[i] = 0;
            R.psize[i] = 0;
        }
        if (i <= R.nparts) R.pc[i] = 0;
        if (i < R.n) {
            if (!keep) R.saving[i] = 0;
            R.pred[i] = -1;
            R.succ[i] = -1;
            R.chain[i] = -1;
            R.mvpos[i] = -1;
            R.cgain[i] = 0;
            R.gseq[i] = 0;
            R.acc0[i] = 0;
            R.dDs[i] = 0;
            R.dDd[i] = 0;
            R.viol[i] = 0;
        }
        if (i < C_N) R.cnt[i] = 0;
        if (i <= R.rounds) R.linked[i] = 0;
    }
}

__global__ void k_rep_nodes(const int32_t *rho, const int32_t *size, const int32_t *singin, int32_t n,
                            long long *psize, int32_t *D0) {
    HP_KERNEL_ENTER();
    GRID_STRIDE(v, (int64_t)n) {
        int32_t p = rho[v];
        atomicAdd((unsigned long long *)&psize[p], (unsigned long long)size[v]);
        if (singin[v]) atomicAdd(&D0[p], singin[v]);
    }
}

// Cut incident hyperedges (|e| >= 2 and more than one part): the only ones
// that add to conn(v, p) for p != rho(v).  Compacted per node, in incidence
// order, for the gain kernels.
// Also counts, for the step's algorithmic bytes, the pins-list entries of
// the level (sum of lambda(e), once per hyperedge: at the entry of its first
// pin), the cut incidence entries and the list entries the gain kernels walk
// for them (sum of lambda(e) over cut entries), into acc[0..2].
__global__ void k_cut_flags(const int32_t *off, const int32_t *pin, const int32_t *inc, const int32_t *inode,
                            const int32_t *lam, int64_t np, int32_t *flag, unsigned long long *acc) {
    HP_KERNEL_ENTER();
    unsigned long long lsum = 0, cuts = 0, clam = 0;
    GRID_STRIDE(t, np) {
        const int32_t e = inc[t];
        const bool listed = off[e + 1] - off[e] >= 2;   // single-pin hyperedges have no pins list
        const int32_t f = (listed && lam[e] >= 2) ? 1 : 0;
        flag[t] = f;
        if (listed && inode[t] == pin[off[e]]) lsum += (unsigned long long)lam[e];
        cuts += (unsigned long long)f;
        if (f) clam += (unsigned long long)lam[e];
    }
    // one update of each counter per CTA (all CTAs hit the same three words)
    __shared__ unsigned long long s_acc[3];
    if (threadIdx.x < 3) s_acc[threadIdx.x] = 0;
    __syncthreads();
    for (int o = 16; o > 0; o >>= 1) {
        lsum += __shfl_down_sync(0xffffffffu, lsum, o);
        cuts += __shfl_down_sync(0xffffffffu, cuts, o);
        clam += __shfl_down_sync(0xffffffffu, clam, o);
    }
    if ((threadIdx.x & 31) == 0 && (lsum | cuts | clam)) {
        atomicAdd(&s_acc[0], lsum);
        atomicAdd(&s_acc[1], cuts);
        atomicAdd(&s_acc[2], clam);
    }
    __syncthreads();
    if (threadIdx.x < 3 && s_acc[threadIdx.x]) atomicAdd(&acc[threadIdx.x], s_acc[threadIdx.x]);
}
__global__ void k_cut_fill(const int32_t *inc, const int32_t *flag, const int32_t *cpos, const int32_t *ioff,
                           int64_t np, int32_t n, int32_t *cut, int32_t *cut_off) {
    HP_KERNEL_ENTER();
    GRID_STRIDE(t, np) {
        if (flag[t]) cut[cpos[t]] = inc[t];
    }
    GRID_STRIDE(v, (int64_t)n + 1) cut_off[v] = cpos[ioff[v]];
}

// candidates: nodes that can spare a cut, by number of cut hyperedges:
// up to GW_DEG a warp each, up to HUB_DEG a CTA each, more a large CTA each
constexpr int32_t HUB_DEG = 1024, GW_DEG = 256;
__global__ void k_candidates(const long long *saving, const int32_t *cut_off, int32_t n, int32_t *list, int32_t *cnt,
                             int32_t *hubs, int32_t *hcnt, int32_t *wlist, int32_t *wcnt) {
    HP_KERNEL_ENTER();
    GRID_STRIDE(v, (int64_t)n) {
        if (saving[v] > 0) {
            const int32_t d = cut_off[v + 1] - cut_off[v];
            if (d > HUB_DEG) hubs[atomicAdd(hcnt, 1)] = (int32_t)v;
            else if (d <= GW_DEG) wlist[atomicAdd(wcnt, 1)] = (int32_t)v;
            else list[atomicAdd(cnt, 1)] = (int32_t)v;
        }
    }
}

// ---------------------------------------------------------------- phases
// Each phase is a strided loop (t0, nt): a kernel runs it over its grid, the
// single-CTA sequence kernels over their block, with a barrier in between.

// sort keys (p_s, gbound - gain, node): ascending = (p_s asc, gain desc, node asc)
__device__ void ph_move_keys(const Moves &M, int32_t m, long long gbound, int gb, int nb, int field, uint64_t *keys,
                             uint32_t *idx, int init_idx, int64_t t0, int64_t nt) {
    STRIDE(i, m, t0, nt) {
        if (init_idx) idx[i] = (uint32_t)i;
        uint32_t k = idx[i];
        uint64_t g = (uint64_t)(gbound - M.gain[k]);
        if (field < 0) keys[i] = ((uint64_t)M.src[k] << (gb + nb)) | (g << nb) | (uint64_t)M.node[k];
        else keys[i] = field == 0 ? (uint64_t)M.node[k] : field == 1 ? g : (uint64_t)M.src[k];
    }
}
// the moves in sorted order, with the size and |in| of each moved node
__device__ void ph_gather(const Moves &M, const uint32_t *idx, int32_t m, const Moves &S, int32_t *pc,
                          const int32_t *size, const int32_t *nin, int32_t *msz, int32_t *mni, int64_t t0, int64_t nt) {
    STRIDE(i, m, t0, nt) {
        uint32_t k = idx[i];
        const int32_t v = M.node[k];
        S.node[i] = v;
        S.src[i] = M.src[k];
        S.dst[i] = M.dst[k];
        S.gain[i] = M.gain[k];
        msz[i] = size[v];
        mni[i] = nin[v];
        atomicAdd(&pc[M.src[k]], 1);
    }
}

struct ChainCtx {
    int32_t window;
    const int32_t *node, *src, *dst, *size, *nin;
    const int32_t *msz, *mni;   // size and |in| of the node of each sorted move
    const long long *gain;
    const int32_t *first;   // [nparts+1]: moves leaving p are [first[p], first[p+1])
    int32_t *pred, *succ, *choice;
    unsigned long long *pen, *minpen;     // general acceptance
    int32_t *accnode;
    unsigned long long *acc[3];           // packed acceptance (penalty < 2^32)
    int32_t *linked;                      // linked[r]: round r linked something
};

// Sec. VI-C: every free chain end picks, among the first `window` moves
// leaving its destination that have no predecessor, the one of maximum
// grade G = gain(m)*10^7 - 10|size(n)-size(m)| - |nin(n)-nin(m)|, earliest on
// ties.  For a chosen move all choosers share gain(m), so the acceptor of
// maximum (G, node id) is the chooser of minimum penalty, then maximum id.
__device__ void ph_choose(const ChainCtx &C, int r, int packed, int32_t m, int64_t t0, int64_t nt) {
    constexpr int B = 4;   // candidates loaded together, ahead of their evaluation
    STRIDE(i0, m, t0, nt) {
        int32_t i = (int32_t)i0;
        C.choice[i] = -1;
        if (!packed) {
            C.minpen[i] = ~0ull;
            C.accnode[i] = -1;
        }
        if (C.succ[i] >= 0) continue;
        const int32_t d = C.dst[i];
        int32_t seen = 0, best = -1;
        __int128 bG = 0;
        unsigned long long bpen = 0;
        const int32_t vi = C.node[i], szi = C.msz[i], nii = C.mni[i];
        const int32_t jend = C.first[d + 1];
        for (int32_t j0 = C.first[d]; j0 < jend && seen < C.window; j0 += B) {
            int32_t pr[B], sz[B], ni[B];
            long long gn[B];
#pragma unroll
            for (int u = 0; u < B; u++) {
                const int32_t j = j0 + u;
                const bool ok = j < jend;
                pr[u] = ok ? C.pred[j] : 0;
                sz[u] = ok ? C.msz[j] : 0;
                ni[u] = ok ? C.mni[j] : 0;
                gn[u] = ok ? C.gain[j] : 0;
            }
#pragma unroll
            for (int u = 0; u < B; u++) {
                const int32_t j = j0 + u;
                if (j >= jend || seen >= C.window) break;
                if (pr[u] >= 0 || j == i) continue;
                seen++;
                const long long ds = (long long)szi - sz[u], di = (long long)nii - ni[u];
                const unsigned long long pen =
                    10ull * (unsigned long long)(ds < 0 ? -ds : ds) + (unsigned long long)(di < 0 ? -di : di);
                const __int128 G = (__int128)gn[u] * 10000000 - (__int128)pen;
                if (best < 0 || G > bG) {
                    best = j;
                    bG = G;
                    bpen = pen;
                }
            }
        }
        C.choice[i] = best;
        C.pen[i] = bpen;
        if (best >= 0 && packed)
            atomicMax(&((r & 1) ? C.acc[1] : C.acc[0])[best],
                      ((0xffffffffull - bpen) << 32) | (unsigned long long)(uint32_t)vi);
    }
}
__device__ void ph_accept_min(const ChainCtx &C, int32_t m, int64_t t0, int64_t nt) {
    STRIDE(i, m, t0, nt) {
        int32_t j = C.choice[i];
        if (j >= 0) atomicMin(&C.minpen[j], C.pen[i]);
    }
}
__device__ void ph_accept_id(const ChainCtx &C, int32_t m, int64_t t0, int64_t nt) {
    STRIDE(i, m, t0, nt) {
        int32_t j = C.choice[i];
        if (j >= 0 && C.pen[i] == C.minpen[j]) atomicMax(&C.accnode[j], C.node[i]);
    }
}
// link the winners; clear the packed slots of the next round
__device__ void ph_link(const ChainCtx &C, int r, int packed, int32_t m, int64_t t0, int64_t nt) {
    STRIDE(i, m, t0, nt) {
        int32_t j = C.choice[i];
        bool won = false;
        if (j >= 0) {
            if (packed)
                won = ((r & 1) ? C.acc[1] : C.acc[0])[j] ==
                      (((0xffffffffull - C.pen[i]) << 32) | (unsigned long long)(uint32_t)C.node[i]);
            else
                won = C.pen[i] == C.minpen[j] && C.accnode[j] == C.node[i];
        }
        if (won) {
            C.pred[j] = (int32_t)i;
            C.succ[i] = j;
            C.linked[r] = 1;
        }
        if (packed) ((r & 1) ? C.acc[0] : C.acc[1])[i] = 0;
    }
}

// One chaining round with one barrier (packed acceptance only).  Round r's
// winners are linked in round r + 1's pass instead of a pass of their own:
// the chooser of a move j won it in round r iff acc_r[j] holds its key, and a
// move j already has a predecessor in round r + 1 iff pred[j] >= 0 (rounds
// before r) or acc_r[j] != 0 (round r: every chosen move gets exactly one
// winner).  The slots rotate over three arrays, round r in acc[r % 3]; the
// pass of round r clears acc[(r + 1) % 3], which the pass of round r - 1 read
// and the pass of round r + 1 fills.  The links of the last round are made by
// ph_link_last.  The result equals the two-pass round above.
__device__ __forceinline__ unsigned long long chain_key(unsigned long long pen, int32_t node) {
    return ((0xffffffffull - pen) << 32) | (unsigned long long)(uint32_t)node;
}
__device__ void ph_round(const ChainCtx &C, int r, int32_t m, int64_t t0, int64_t nt) {
    constexpr int B = 4;
    unsigned long long *accr = C.acc[r % 3], *accp = C.acc[(r + 2) % 3], *accn = C.acc[(r + 1) % 3];
    STRIDE(i0, m, t0, nt) {
        const int32_t i = (int32_t)i0;
        bool taken_end = C.succ[i] >= 0;
        if (r > 0) {
            const int32_t j = C.choice[i];
            if (j >= 0 && accp[j] == chain_key(C.pen[i], C.node[i])) {
                C.pred[j] = i;
                C.succ[i] = j;
                taken_end = true;
            }
        }
        accn[i] = 0;
        C.choice[i] = -1;
        if (taken_end) continue;
        const int32_t d = C.dst[i];
        int32_t seen = 0, best = -1;
        __int128 bG = 0;
        unsigned long long bpen = 0;
        const int32_t szi = C.msz[i], nii = C.mni[i];
        const int32_t jend = C.first[d + 1];
        for (int32_t j0 = C.first[d]; j0 < jend && seen < C.window; j0 += B) {
            bool tk[B];
            int32_t sz[B], ni[B];
            long long gn[B];
#pragma unroll
            for (int u = 0; u < B; u++) {
                const int32_t j = j0 + u;
                const bool ok = j < jend;
                tk[u] = ok ? (C.pred[j] >= 0 || (r > 0 && accp[j] != 0ull)) : true;
                sz[u] = ok ? C.msz[j] : 0;
                ni[u] = ok ? C.mni[j] : 0;
                gn[u] = ok ? C.gain[j] : 0;
            }
#pragma unroll
            for (int u = 0; u < B; u++) {
                const int32_t j = j0 + u;
                if (j >= jend || seen >= C.window) break;
                if (tk[u] || j == i) continue;
                seen++;
                const long long ds = (long long)szi - sz[u], di = (long long)nii - ni[u];
                const unsigned long long pen =
                    10ull * (unsigned long long)(ds < 0 ? -ds : ds) + (unsigned long long)(di < 0 ? -di : di);
                const __int128 G = (__int128)gn[u] * 10000000 - (__int128)pen;
                if (best < 0 || G > bG) {
                    best = j;
                    bG = G;
                    bpen = pen;
                }
            }
        }
        C.choice[i] = best;
        C.pen[i] = bpen;
        if (best >= 0) {
            atomicMax(&accr[best], chain_key(bpen, C.node[i]));
            C.linked[r] = 1;
        }
    }
}
// the links of round r, the last round run (nothing when it chose nothing)
__device__ void ph_link_last(const ChainCtx &C, int r, int32_t m, int64_t t0, int64_t nt) {
    const unsigned long long *accr = C.acc[r % 3];
    STRIDE(i0, m, t0, nt) {
        const int32_t i = (int32_t)i0, j = C.choice[i];
        if (j >= 0 && accr[j] == chain_key(C.pen[i], C.node[i])) {
            C.pred[j] = i;
            C.succ[i] = j;
        }
    }
}

struct SeqCtx {
    const int32_t *node, *pred, *succ;
    const long long *gain;
    int32_t *chain, *pos, *clen;
    long long *cgain;
    uint32_t *err;
};
__device__ void ph_path_heads(const SeqCtx &S, int32_t m, int64_t t0, int64_t nt) {
    STRIDE(i0, m, t0, nt) {
        int32_t i = (int32_t)i0;
        if (S.pred[i] >= 0) continue;
        long long g = 0;
        int32_t k = 0;
        for (int32_t j = i; j >= 0; j = S.succ[j]) {
            if (k > m) {
                atomicOr(S.err, E_TIMEOUT);
                break;
            }
            S.chain[j] = i;
            S.pos[j] = k++;
            g += S.gain[j];
        }
        S.clen[i] = k;
        S.cgain[i] = g;
    }
}
// moves left unassigned lie on cycles; the member of smallest node id heads it
__device__ void ph_cycle_heads(const SeqCtx &S, int32_t m, int64_t t0, int64_t nt) {
    STRIDE(i0, m, t0, nt) {
        int32_t i = (int32_t)i0;
        if (S.chain[i] >= 0) continue;
        int32_t mn = S.node[i], k = 0;
        for (int32_t j = S.succ[i]; j != i; j = S.succ[j]) {
            if (j < 0 || ++k > m) {
                atomicOr(S.err, E_INTERNAL);
                mn = -1;
                break;
            }
            mn = min(mn, S.node[j]);
        }
        if (mn != S.node[i]) continue;
        long long g = 0;
        int32_t c = 0, j = i;
        do {
            S.chain[j] = i;
            S.pos[j] = c++;
            g += S.gain[j];
            j = S.succ[j];
        } while (j != i && c <= m);
        S.clen[i] = c;
        S.cgain[i] = g;
    }
}
__device__ void ph_head_collect(const SeqCtx &S, int32_t m, uint32_t *heads, int32_t *nh, int64_t t0, int64_t nt) {
    STRIDE(i, m, t0, nt) {
        if (S.chain[i] == (int32_t)i) heads[atomicAdd(nh, 1)] = (uint32_t)i;
    }
}
// key (cgbound - chain gain, head node): ascending = (total gain desc, head node asc)
__device__ void ph_head_keys(const uint32_t *heads, int32_t nh, const long long *cgain, const int32_t *node,
                             long long cgbound, int nb, int field, uint64_t *keys, int64_t t0, int64_t nt) {
    STRIDE(k, nh, t0, nt) {
        uint32_t h = heads[k];
        uint64_t gk = (uint64_t)(cgbound - cgain[h]);
        if (field < 0) keys[k] = (gk << nb) | (uint64_t)node[h];
        else keys[k] = field == 0 ? (uint64_t)node[h] : gk;
    }
}
__device__ void ph_chain_lens(const uint32_t *heads, int32_t nh, const int32_t *clen, int64_t cap, int32_t *lens,
                              int64_t t0, int64_t nt) {
    STRIDE(k, cap, t0, nt) lens[k] = k < nh ? clen[heads[k]] : 0;
}
__device__ void ph_chain_start(const uint32_t *heads, int32_t nh, const int32_t *starts, int32_t *cstart, int64_t t0,
                               int64_t nt) {
    STRIDE(k, nh, t0, nt) cstart[heads[k]] = starts[k];
}
__device__ void ph_seq_pos(const int32_t *chain, const int32_t *pos, const int32_t *cstart, int32_t m,
                           const int32_t *node, int32_t *seqmove, int32_t *mvpos, int64_t t0, int64_t nt) {
    STRIDE(i, m, t0, nt) {
        int32_t k = cstart[chain[i]] + pos[i];
        seqmove[k] = (int32_t)i;
        mvpos[node[i]] = k;
    }
}

// Sec. VI-D: two capacity entries per move k, in sequence order: at p_s
// (-size, dD_s) and at p_d (+size, dD_d); sorted stably by part, each part's
// entries are walked in sequence order and each change of its validity is
// recorded at the move that caused it.
struct ValCtx {
    const int32_t *seqmove, *size, *singin, *dDs, *dDd, *D0;
    const unsigned long long *gseq;
    Moves S;
    const long long *psize;
    uint32_t *vkey, *vidx;
    long long *vsz;
    int32_t *vdd, *viol;
    int32_t omega, delta;
    long long *gsz, *gdd, *esz, *edd;  // [2m] events in part order; their exclusive prefix sums
    int32_t *vhead;                    // [nparts] first event of each part
};
__device__ void ph_val_entries(const ValCtx &V, int32_t m, int64_t t0, int64_t nt) {
    STRIDE(k, m, t0, nt) {
        int32_t i = V.seqmove[k];
        int32_t v = V.S.node[i];
        long long sz = V.size[v];
        V.vkey[2 * k] = (uint32_t)V.S.src[i];
        V.vidx[2 * k] = (uint32_t)(2 * k);
        V.vsz[2 * k] = -sz;
        V.vdd[2 * k] = V.dDs[k] - V.singin[v];
        V.vkey[2 * k + 1] = (uint32_t)V.S.dst[i];
        V.vidx[2 * k + 1] = (uint32_t)(2 * k + 1);
        V.vsz[2 * k + 1] = sz;
        V.vdd[2 * k + 1] = V.dDd[k] + V.singin[v];
    }
}
// Validity of every prefix (Sec. VI-D) from the c = 2m capacity events
// sorted by part (stably, so in sequence order within a part).  A part's
// running size and distinct-inbound count after each of its events are
// global prefix sums minus the prefix at the part's first event; every event
// at which the part turns valid or invalid adds -1 / +1 to the violation
// count of its move.
__device__ void ph_val_gather(const ValCtx &V, int32_t c, int64_t t0, int64_t nt) {
    STRIDE(j, c, t0, nt) {
        const uint32_t x = V.vidx[j];
        V.gsz[j] = V.vsz[x];
        V.gdd[j] = V.vdd[x];
        const uint32_t p = V.vkey[j];
        if (j == 0 || V.vkey[j - 1] != p) V.vhead[p] = (int32_t)j;
    }
}
__device__ void ph_val_trans(const ValCtx &V, int32_t c, int64_t t0, int64_t nt) {
    STRIDE(j, c, t0, nt) {
        const uint32_t p = V.vkey[j];
        const int32_t h = V.vhead[p];
        const long long bs = V.psize[p] + (V.esz[j] - V.esz[h]), bd = (long long)V.D0[p] + (V.edd[j] - V.edd[h]);
        const long long as = bs + V.gsz[j], ad = bd + V.gdd[j];
        const bool vb = bs <= V.omega && bd <= V.delta, va = as <= V.omega && ad <= V.delta;
        if (vb != va) atomicAdd(&V.viol[V.vidx[j] >> 1], va ? -1 : 1);
    }
}
__device__ int32_t ph_initial_bad(const long long *psize, const int32_t *D0, int32_t nparts, int32_t omega,
                                  int32_t delta, int64_t t0, int64_t nt) {
    int32_t c = 0;
    STRIDE(p, nparts, t0, nt) c += (psize[p] > omega || D0[p] > delta) ? 1 : 0;
    return c;
}
__device__ void ph_apply(const int32_t *seqmove, const int32_t *node, const int32_t *dst, int32_t L, int32_t *rho,
                         int64_t t0, int64_t nt) {
    STRIDE(k, L, t0, nt) {
        int32_t i = seqmove[k];
        rho[node[i]] = dst[i];
    }
}

// ---- block-level helpers of the single-CTA kernels (blockDim = SEQ_T)
// the same for int64 values, in place allowed (in == out)
__device__ void block_scan_excl_ll(const long long *in, long long *out, int64_t n, long long *s_tmp) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    long long carry = 0;
    for (int64_t base = 0; base < n; base += blockDim.x) {
        int64_t i = base + threadIdx.x;
        long long x = i < n ? in[i] : 0, inc = x;
        for (int o = 1; o < 32; o <<= 1) {
            long long u = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += u;
        }
        if (lane == 31) s_tmp[wid] = inc;
        __syncthreads();
        if (wid == 0) {
            long long y = lane < nw ? s_tmp[lane] : 0, yi = y;
            for (int o = 1; o < 32; o <<= 1) {
                long long u = __shfl_up_sync(0xffffffffu, yi, o);
                if (lane >= o) yi += u;
            }
            if (lane < nw) s_tmp[lane] = yi - y;
            if (lane == nw - 1) s_tmp[32] = yi;
        }
        __syncthreads();
        if (i < n) out[i] = carry + s_tmp[wid] + inc - x;
        carry += s_tmp[32];
        __syncthreads();
    }
}

// best prefix (Sec. VI-D): max cumulative gain over prefixes with zero
// invalid parts, longest on ties; one CTA of 1024 threads
__device__ void best_prefix_block(const unsigned long long *gseq, const int32_t *violc, int32_t m, int32_t bad0,
                                  int32_t *best_len, long long *best_gain) {
    __shared__ long long s_g[32];
    __shared__ int32_t s_k[32];
    __shared__ long long s_carry_g;
    __shared__ int32_t s_carry_v;
    if (threadIdx.x == 0) {
        s_carry_g = 0;
        s_carry_v = bad0;
    }
    __syncthreads();
    long long bestg = 0;
    int32_t bestk = 0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int32_t base = 0; base < m; base += 1024) {
        int32_t k = base + threadIdx.x;
        long long g = k < m ? (long long)gseq[k] : 0;
        int32_t dv = k < m ? violc[k] : 0;
        long long gi = g;
        int32_t vi = dv;
        for (int o = 1; o < 32; o <<= 1) {
            long long ug = __shfl_up_sync(0xffffffffu, gi, o);
            int32_t uv = __shfl_up_sync(0xffffffffu, vi, o);
            if (lane >= o) {
                gi += ug;
                vi += uv;
            }
        }
        if (lane == 31) {
            s_g[wid] = gi;
            s_k[wid] = vi;
        }
        __syncthreads();
        if (wid == 0) {
            long long x = s_g[lane];
            int32_t y = s_k[lane];
            long long xi = x;
            int32_t yi = y;
            for (int o = 1; o < 32; o <<= 1) {
                long long ux = __shfl_up_sync(0xffffffffu, xi, o);
                int32_t uy = __shfl_up_sync(0xffffffffu, yi, o);
                if (lane >= o) {
                    xi += ux;
                    yi += uy;
                }
            }
            s_g[lane] = xi - x;
            s_k[lane] = yi - y;
        }
        __syncthreads();
        long long cum = s_carry_g + s_g[wid] + gi;
        int32_t vio = s_carry_v + s_k[wid] + vi;
        if (k < m && vio == 0 && cum >= bestg) {
            bestg = cum;
            bestk = k + 1;
        }
        __syncthreads();
        if (threadIdx.x == 1023) {
            s_carry_g = cum;
            s_carry_v = vio;
        }
        __syncthreads();
    }
    for (int o = 16; o > 0; o >>= 1) {
        long long og = __shfl_down_sync(0xffffffffu, bestg, o);
        int32_t ok = __shfl_down_sync(0xffffffffu, bestk, o);
        if (og > bestg || (og == bestg && ok > bestk)) {
            bestg = og;
            bestk = ok;
        }
    }
    if (lane == 0) {
        s_g[wid] = bestg;
        s_k[wid] = bestk;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < 32; k++)
            if (s_g[k] > bestg || (s_g[k] == bestg && s_k[k] > bestk)) {
                bestg = s_g[k];
                bestk = s_k[k];
            }
        *best_gain = bestg;
        *best_len = bestg > 0 ? bestk : 0;
    }
    __syncthreads();
}

// ---------------------------------------------------------------- multi-kernel path
__global__ void k_move_keys(const Moves M, const int32_t *cntp, long long gbound, int gb, int nb, int field,
                            uint64_t *keys, uint32_t *idx, int init_idx) {
    HP_KERNEL_ENTER();
    ph_move_keys(M, *cntp, gbound, gb, nb, field, keys, idx, init_idx, G_T0, G_NT);
}
__global__ void k_gather_moves(const Moves M, const uint32_t *idx, const int32_t *cntp, Moves S, int32_t *pc,
                               const int32_t *size, const int32_t *nin, int32_t *msz, int32_t *mni) {
    HP_KERNEL_ENTER();
    ph_gather(M, idx, *cntp, S, pc, size, nin, msz, mni, G_T0, G_NT);
}
__global__ void k_choose(ChainCtx C, const int32_t *mcount, int r, int packed) {
    HP_KERNEL_ENTER();
    if (r > 0 && !C.linked[r - 1]) return;
    ph_choose(C, r, packed, *mcount, G_T0, G_NT);
}
__global__ void k_accept_min(ChainCtx C, const int32_t *mcount, int r) {
    HP_KERNEL_ENTER();
    if (r > 0 && !C.linked[r - 1]) return;
    ph_accept_min(C, *mcount, G_T0, G_NT);
}
__global__ void k_accept_id(ChainCtx C, const int32_t *mcount, int r) {
    HP_KERNEL_ENTER();
    if (r > 0 && !C.linked[r - 1]) return;
    ph_accept_id(C, *mcount, G_T0, G_NT);
}
__global__ void k_link(ChainCtx C, const int32_t *mcount, int r, int packed) {
    HP_KERNEL_ENTER();
    if (r > 0 && !C.linked[r - 1]) return;
    ph_link(C, r, packed, *mcount, G_T0, G_NT);
}

__global__ void k_path_heads(SeqCtx S, const int32_t *mcount) { HP_KERNEL_ENTER(); ph_path_heads(S, *mcount, G_T0, G_NT); }
__global__ void k_cycle_heads(SeqCtx S, const int32_t *mcount) { HP_KERNEL_ENTER(); ph_cycle_heads(S, *mcount, G_T0, G_NT); }
__global__ void k_head_collect(SeqCtx S, const int32_t *mcount, uint32_t *heads, int32_t *nh) {
    HP_KERNEL_ENTER();
    ph_head_collect(S, *mcount, heads, nh, G_T0, G_NT);
}
__global__ void k_head_keys(const uint32_t *heads, const int32_t *nh, const long long *cgain, const int32_t *node,
                            long long cgbound, int nb, int field, uint64_t *keys) {
    HP_KERNEL_ENTER();
    ph_head_keys(heads, *nh, cgain, node, cgbound, nb, field, keys, G_T0, G_NT);
}
__global__ void k_chain_lens(const uint32_t *heads, const int32_t *nh, const int32_t *clen, int32_t cap,
                             int32_t *lens) {
    HP_KERNEL_ENTER();
    ph_chain_lens(heads, *nh, clen, cap, lens, G_T0, G_NT);
}
__global__ void k_chain_start(const uint32_t *heads, const int32_t *nh, const int32_t *starts, int32_t *cstart) {
    HP_KERNEL_ENTER();
    ph_chain_start(heads, *nh, starts, cstart, G_T0, G_NT);
}
__global__ void k_seq_pos(const int32_t *chain, const int32_t *pos, const int32_t *cstart, const int32_t *mcount,
                          const int32_t *node, int32_t *seqmove, int32_t *mvpos) {
    HP_KERNEL_ENTER();
    ph_seq_pos(chain, pos, cstart, *mcount, node, seqmove, mvpos, G_T0, G_NT);
}
__global__ void k_val_entries(ValCtx V, const int32_t *mcount, int32_t *nv) {
    HP_KERNEL_ENTER();
    const int32_t m = *mcount;
    if (blockIdx.x == 0 && threadIdx.x == 0) *nv = 2 * m;
    ph_val_entries(V, m, G_T0, G_NT);
}
__global__ void k_val_gather(ValCtx V, const int32_t *nv) { HP_KERNEL_ENTER(); ph_val_gather(V, *nv, G_T0, G_NT); }
__global__ void k_val_trans(ValCtx V, const int32_t *nv) { HP_KERNEL_ENTER(); ph_val_trans(V, *nv, G_T0, G_NT); }
__global__ void k_initial_bad(const long long *psize, const int32_t *D0, int32_t nparts, int32_t omega, int32_t delta,
                              int32_t *bad) {
    HP_KERNEL_ENTER();
    int32_t c = ph_initial_bad(psize, D0, nparts, omega, delta, G_T0, G_NT);
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(bad, c);
}
__global__ void __launch_bounds__(1024) k_best_prefix(const unsigned long long *gseq, const int32_t *violc,
                                                      const int32_t *mcount, const int32_t *bad0, int32_t *best_len,
                                                      long long *best_gain) {
    HP_KERNEL_ENTER();
    best_prefix_block(gseq, violc, *mcount, *bad0, best_len, best_gain);
}
__global__ void k_apply(const int32_t *seqmove, const int32_t *node, const int32_t *dst, const int32_t *lenp,
                        int32_t *rho) {
    HP_KERNEL_ENTER();
    ph_apply(seqmove, node, dst, *lenp, rho, G_T0, G_NT);
}

// ---------------------------------------------------------------- cluster path (M <= sq_max<uint64_t>())
// Sort of the moves, chaining rounds, chain order and sequence positions of
// one repetition by one thread-block cluster (hp_cluster.cuh): every phase is
// a strided loop over the cluster's threads on the global arrays (L2
// resident at these sizes), separated by cluster barriers; the two sorts are
// cluster radix sorts.  Eight times the threads of one CTA, so the latency of
// each phase's global loads is spread over 8 SMs.
static_assert(SQ_T == SEQ_T, "cluster CTA size");
constexpr int32_t SEQ_CLUSTER_M = 4096;   // moves of a larger level sequenced by one cluster
static_assert(SMALL_LEVEL <= sq_max<uint64_t>() && 2 * SMALL_LEVEL <= sq_max<uint32_t>(),
              "a small level's moves fit the cluster sorts");

struct ClusterSeqArgs {
    Moves M, S;
    uint64_t *keys, *hkeys;
    uint32_t *idx, *heads;
    int32_t *first, *lens, *starts, *cstart, *seqmove, *mvpos, *cnt;
    ChainCtx C;
    SeqCtx Q;
    int32_t nparts, rounds, packed, gb, nb, sb, cgb;
    long long gbound, cgbound;
};

// first[p] = number of sorted moves leaving a part below p, for p in [0, nparts]
__device__ void ph_first_of(const int32_t *src, int32_t m, int32_t nparts, int32_t *first, int64_t t0, int64_t nt) {
    STRIDE(p, (int64_t)nparts + 1, t0, nt) {
        int32_t a = 0, b = m;
        while (a < b) {
            const int32_t mid = (a + b) >> 1;
            if (src[mid] < (int32_t)p) a = mid + 1;
            else b = mid;
        }
        first[p] = a;
    }
}

__global__ void __cluster_dims__(SQ_CS, 1, 1) __launch_bounds__(SEQ_T) k_seq_cluster(ClusterSeqArgs A) {
    HP_KERNEL_ENTER();
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_wc[32 * 256];
    __shared__ uint32_t s_tot[256];
    __shared__ uint32_t s_base[512];
    __shared__ int32_t s_tmp[40];
    __shared__ int32_t s_part;
    __shared__ long long s_ll[40];
    cg::cluster_group cl = cg::this_cluster();
    const int32_t m = A.cnt[C_MOVES];
    if (m == 0 || m > sq_max<uint64_t>()) return;   // uniform: no CTA of the cluster runs on
    const int64_t t0 = (int64_t)cl.block_rank() * blockDim.x + threadIdx.x, nt = (int64_t)SQ_CS * blockDim.x;
    const SqBuf<uint64_t> B(smem);
    // key widths from this repetition's moves
    long long gmx = 0, smx = 0, nmx = 0;
    STRIDE(i, m, t0, nt) {
        gmx = max(gmx, A.M.gain[i]);
        smx = max(smx, (long long)A.M.src[i]);
        nmx = max(nmx, (long long)A.M.node[i]);
    }
    cluster_max3_ll(cl, gmx, smx, nmx, s_ll);
    const int gb = dev_bits((unsigned long long)gmx), nb = dev_bits((unsigned long long)nmx),
              sb = dev_bits((unsigned long long)smx);
    // sort (p_s asc, gain desc, node asc)
    if (sb + gb + nb <= 64) {
        ph_move_keys(A.M, m, gmx, gb, nb, -1, A.keys, A.idx, 1, t0, nt);
        cl.sync();
        cluster_radix_sort<uint64_t>(cl, A.keys, A.idx, m, (sb + gb + nb + 7) / 8, B, s_wc, s_tot, s_base);
    } else {
        const int fb[3] = {A.nb, A.gb, A.sb};
        for (int f = 0; f < 3; f++) {
            ph_move_keys(A.M, m, A.gbound, A.gb, A.nb, f, A.keys, A.idx, f == 0, t0, nt);
            cl.sync();
            cluster_radix_sort<uint64_t>(cl, A.keys, A.idx, m, (fb[f] + 7) / 8, B, s_wc, s_tot, s_base);
        }
    }
    // the moves in sorted order, with the size and |in| of each moved node
    STRIDE(i, m, t0, nt) {
        const uint32_t k = A.idx[i];
        const int32_t v = A.M.node[k];
        A.S.node[i] = v;
        A.S.src[i] = A.M.src[k];
        A.S.dst[i] = A.M.dst[k];
        A.S.gain[i] = A.M.gain[k];
        const_cast<int32_t *>(A.C.msz)[i] = A.C.size[v];
        const_cast<int32_t *>(A.C.mni)[i] = A.C.nin[v];
    }
    cl.sync();
    ph_first_of(A.S.src, m, A.nparts, A.first, t0, nt);
    cl.sync();
    // chaining rounds (Sec. VI-C)
    for (int rr = 0; rr < A.rounds; rr++) {
        if (rr > 0 && !*(volatile int32_t *)&A.C.linked[rr - 1]) break;
        if (A.packed) {
            ph_round(A.C, rr, m, t0, nt);
            cl.sync();
            continue;
        }
        ph_choose(A.C, rr, A.packed, m, t0, nt);
        cl.sync();
        ph_accept_min(A.C, m, t0, nt);
        cl.sync();
        ph_accept_id(A.C, m, t0, nt);
        cl.sync();
        ph_link(A.C, rr, A.packed, m, t0, nt);
        cl.sync();
    }
    if (A.packed && A.rounds > 0 && *(volatile int32_t *)&A.C.linked[A.rounds - 1]) {
        ph_link_last(A.C, A.rounds - 1, m, t0, nt);
        cl.sync();
    }
    // chains, ordered by (total gain desc, head node asc)
    ph_path_heads(A.Q, m, t0, nt);
    cl.sync();
    ph_cycle_heads(A.Q, m, t0, nt);
    cl.sync();
    ph_head_collect(A.Q, m, A.heads, &A.cnt[C_NH], t0, nt);
    cl.sync();
    const int32_t nh = *(volatile int32_t *)&A.cnt[C_NH];
    long long cmx = 0;
    STRIDE(k, nh, t0, nt) cmx = max(cmx, A.Q.cgain[A.heads[k]]);
    cmx = cluster_max_ll(cl, cmx, s_ll);
    const int cgb = dev_bits((unsigned long long)cmx);
    if (cgb + nb <= 64) {
        ph_head_keys(A.heads, nh, A.Q.cgain, A.S.node, cmx, nb, -1, A.hkeys, t0, nt);
        cl.sync();
        cluster_radix_sort<uint64_t>(cl, A.hkeys, A.heads, nh, (cgb + nb + 7) / 8, B, s_wc, s_tot, s_base);
    } else {
        for (int f = 0; f < 2; f++) {
            ph_head_keys(A.heads, nh, A.Q.cgain, A.S.node, A.cgbound, A.nb, f, A.hkeys, t0, nt);
            cl.sync();
            cluster_radix_sort<uint64_t>(cl, A.hkeys, A.heads, nh, ((f == 0 ? A.nb : A.cgb) + 7) / 8, B, s_wc,
                                         s_tot, s_base);
        }
    }
    ph_chain_lens(A.heads, nh, A.Q.clen, nh, A.lens, t0, nt);
    cl.sync();
    cluster_scan_excl<int32_t>(cl, A.lens, A.starts, nh, s_tmp, &s_part);
    ph_chain_start(A.heads, nh, A.starts, A.cstart, t0, nt);
    cl.sync();
    ph_seq_pos(A.Q.chain, A.Q.pos, A.cstart, m, A.S.node, A.seqmove, A.mvpos, t0, nt);
    cl.sync();   // no CTA leaves while another may still read its shared memory
}

// validity of every prefix, best prefix, apply
__global__ void __launch_bounds__(SEQ_T) k_val_small(ValCtx V, int32_t *cnt, int32_t nparts, int sb, long long *bgain,
                                                     int32_t *rho) {
    HP_KERNEL_ENTER();
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_wc[32 * 256];
    __shared__ uint32_t s_hist[256 + 33];
    __shared__ int32_t s_tmp[40];
    __shared__ long long s_ll[40];
    const int32_t m = cnt[C_MOVES];
    if (m == 0 || m > SMALLM) return;
    const int64_t t0 = threadIdx.x, nt = blockDim.x;
    ph_val_entries(V, m, t0, nt);
    block_radix_sort<uint32_t>(V.vkey, V.vidx, 2 * m, (sb + 7) / 8, 2 * SMALLM, smem, s_wc, s_hist);
    __syncthreads();
    ph_val_gather(V, 2 * m, t0, nt);
    __syncthreads();
    block_scan_excl_ll(V.gsz, V.esz, 2 * m, s_ll);
    block_scan_excl_ll(V.gdd, V.edd, 2 * m, s_ll);
    ph_val_trans(V, 2 * m, t0, nt);
    int32_t bad = block_sum(ph_initial_bad(V.psize, V.D0, nparts, V.omega, V.delta, t0, nt), s_tmp);
    __syncthreads();
    best_prefix_block(V.gseq, V.viol, m, bad, &cnt[C_APPLIED], bgain);
    const int32_t L = *(volatile int32_t *)&cnt[C_APPLIED];
    ph_apply(V.seqmove, V.S.node, V.S.dst, L, rho, t0, nt);
}

// The same on one thread-block cluster, for up to sq_max<uint32_t>() / 2
// moves: events, cluster radix sort by part, the two prefix sums, the
// validity transitions, the count of invalid parts, the best prefix and the
// apply, separated by cluster barriers.
__global__ void __cluster_dims__(SQ_CS, 1, 1) __launch_bounds__(SQ_T)
    k_val_cluster(ValCtx V, int32_t *cnt, int32_t nparts, int sb, long long *bgain, int32_t *rho) {
    HP_KERNEL_ENTER();
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_wc[32 * 256];
    __shared__ uint32_t s_tot[256];
    __shared__ uint32_t s_base[512];
    __shared__ long long s_ll[40];
    __shared__ int32_t s_tmp[40];
    __shared__ long long s_part;
    __shared__ int32_t s_ipart;
    __shared__ long long s_bg[32];
    __shared__ int32_t s_bk[32];
    cg::cluster_group cl = cg::this_cluster();
    const int32_t m = cnt[C_MOVES];
    if (m == 0 || 2 * (int64_t)m > sq_max<uint32_t>()) return;   // uniform over the cluster
    const int r = (int)cl.block_rank(), t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
    const int64_t t0 = (int64_t)r * blockDim.x + t, nt = (int64_t)SQ_CS * blockDim.x;
    const int32_t c = 2 * m;
    ph_val_entries(V, m, t0, nt);
    cl.sync();
    cluster_radix_sort<uint32_t>(cl, V.vkey, V.vidx, c, (sb + 7) / 8, SqBuf<uint32_t>(smem), s_wc, s_tot, s_base);
    ph_val_gather(V, c, t0, nt);
    cl.sync();
    cluster_scan_excl<long long>(cl, V.gsz, V.esz, c, s_ll, &s_part);
    cluster_scan_excl<long long>(cl, V.gdd, V.edd, c, s_ll, &s_part);
    ph_val_trans(V, c, t0, nt);
    const int32_t bad0 = cluster_sum_i32(cl, ph_initial_bad(V.psize, V.D0, nparts, V.omega, V.delta, t0, nt), s_tmp,
                                         &s_ipart);
    // best prefix (Sec. VI-D): the largest cumulative gain over prefixes with
    // no invalid part, the longest on ties; this CTA takes moves [lo, hi)
    const int32_t chunk = (m + SQ_CS - 1) / SQ_CS, lo = min(m, r * chunk), hi = min(m, lo + chunk);
    long long gl = 0;
    int32_t vl = 0;
    for (int32_t k = lo + t; k < hi; k += blockDim.x) {
        gl += (long long)V.gseq[k];
        vl += V.viol[k];
    }
    gl = block_sum_ll(gl, s_ll);
    vl = block_sum(vl, s_tmp);
    if (t == 0) {
        s_ll[36] = gl;
        s_ll[37] = vl;
    }
    cl.sync();
    long long gc = 0, vc = bad0;   // sums over the moves before lo
    for (int q = 0; q < r; q++) {
        const long long *o = cl.map_shared_rank(s_ll, q);
        gc += o[36];
        vc += o[37];
    }
    long long bestg = 0;
    int32_t bestk = 0;
    for (int32_t base = lo; base < hi; base += blockDim.x) {
        const int32_t k = base + t;
        const long long g = k < hi ? (long long)V.gseq[k] : 0;
        const long long dv = k < hi ? V.viol[k] : 0;
        long long gi = g, vi = dv;
        for (int o = 1; o < 32; o <<= 1) {
            const long long ug = __shfl_up_sync(0xffffffffu, gi, o), uv = __shfl_up_sync(0xffffffffu, vi, o);
            if (lane >= o) {
                gi += ug;
                vi += uv;
            }
        }
        if (lane == 31) {
            s_ll[wid] = gi;
            s_bg[wid] = vi;
        }
        __syncthreads();
        if (wid == 0) {
            const long long x = lane < nw ? s_ll[lane] : 0, y = lane < nw ? s_bg[lane] : 0;
            long long xi = x, yi = y;
            for (int o = 1; o < 32; o <<= 1) {
                const long long ux = __shfl_up_sync(0xffffffffu, xi, o), uy = __shfl_up_sync(0xffffffffu, yi, o);
                if (lane >= o) {
                    xi += ux;
                    yi += uy;
                }
            }
            if (lane < nw) {
                s_ll[lane] = xi - x;
                s_bg[lane] = yi - y;
            }
            if (lane == nw - 1) {
                s_ll[32] = xi;
                s_ll[33] = yi;
            }
        }
        __syncthreads();
        const long long cum = gc + s_ll[wid] + gi, vio = vc + s_bg[wid] + vi;
        if (k < hi && vio == 0 && cum >= bestg) {
            bestg = cum;
            bestk = k + 1;
        }
        gc += s_ll[32];
        vc += s_ll[33];
        __syncthreads();
    }
    for (int o = 16; o > 0; o >>= 1) {
        const long long og = __shfl_down_sync(0xffffffffu, bestg, o);
        const int32_t ok = __shfl_down_sync(0xffffffffu, bestk, o);
        if (og > bestg || (og == bestg && ok > bestk)) {
            bestg = og;
            bestk = ok;
        }
    }
    if (lane == 0) {
        s_bg[wid] = bestg;
        s_bk[wid] = bestk;
    }
    __syncthreads();
    if (t == 0) {
        for (int k = 1; k < nw; k++)
            if (s_bg[k] > bestg || (s_bg[k] == bestg && s_bk[k] > bestk)) {
                bestg = s_bg[k];
                bestk = s_bk[k];
            }
        s_ll[38] = bestg;
        s_ll[39] = bestk;
    }
    cl.sync();
    if (r == 0 && t == 0) {
        for (int q = 1; q < SQ_CS; q++) {
            const long long *o = cl.map_shared_rank(s_ll, q);
            if (o[38] > bestg || (o[38] == bestg && o[39] > bestk)) {
                bestg = o[38];
                bestk = (int32_t)o[39];
            }
        }
        *bgain = bestg;
        cnt[C_APPLIED] = bestg > 0 ? bestk : 0;
    }
    cl.sync();
    const int32_t L = *(volatile int32_t *)&cnt[C_APPLIED];
    ph_apply(V.seqmove, V.S.node, V.S.dst, L, rho, t0, nt);
    cl.sync();   // no CTA leaves while another may still read its shared memory
}

// ---------------------------------------------------------------- in-sequence gains
// Per hyperedge e with moved pins: its moved pins in sequence order; the
// running pins(p,e) / pins_in(p,e) of the parts they touch start from the
// pins list.  A move that empties e in p_s spares w(e), one that enters an
// empty p_d costs w(e) (Eq. 14-15 read as the exact change of connectivity);
// an inbound count crossing 1 -> 0 at p_s or 0 -> 1 at p_d changes the
// distinct-inbound count of that part at that move (Sec. VI-D).
struct SeqSim {
    const int32_t *off, *pin, *nsrc, *w, *mvpos, *seqmove, *src, *dst;
    Plist PL;
    unsigned long long *gseq;
    int32_t *dDs, *dDd;
};

__device__ __forceinline__ int32_t plist_find(const Plist &PL, int32_t a, int32_t lam, int32_t p) {
    int32_t lo = 0, hi = lam;
    while (lo < hi) {
        int32_t mid = (lo + hi) >> 1;
        if (PL.p[a + mid] < p) lo = mid + 1;
        else hi = mid;
    }
    return (lo < lam && PL.p[a + lo] == p) ? a + lo : -1;
}

// group of G threads; buffers: bk/bd/ord >= |e|, tp/tc/tci >= 2|e|.
// The running counts are not simulated move by move: the move at sequence
// rank r sees pins(p,e) = the pins list's count + (moves of ranks < r into p)
// - (moves of ranks < r out of p), and pins_in(p,e) the same over the moves
// of destination pins, so every rank is evaluated at once (threads over
// ranks, each counting over the ranks before it in shared memory).
template <int G>
__device__ void inseq_edge(const SeqSim &Q, int32_t e, int gt, int32_t *bk, int32_t *bd, int32_t *ord, int32_t *tp,
                           int32_t *tc, int32_t *tci, int32_t *g_cnt) {
    const int32_t a = Q.off[e], b = Q.off[e + 1], dst0 = a + Q.nsrc[e];
    if (gt == 0) *g_cnt = 0;
    gsync<G>();
    for (int32_t j = a + gt; j < b; j += G) {
        int32_t k = Q.mvpos[Q.pin[j]];
        if (k >= 0) {
            int32_t s = atomicAdd(g_cnt, 1);
            bk[s] = k;
            bd[s] = j >= dst0;
        }
    }
    gsync<G>();
    const int32_t c = *(volatile int32_t *)g_cnt;
    if (c == 0) {
        gsync<G>();
        return;
    }
    for (int32_t i = gt; i < c; i += G) {
        int32_t k = bk[i], r = 0;
        for (int32_t t = 0; t < c; t++) r += bk[t] < k;
        ord[r] = i;
    }
    gsync<G>();
    // by rank: source part, destination part, destination-pin flag
    int32_t *rs = tp, *rd = tp + c, *rf = tc;
    for (int32_t r = gt; r < c; r += G) {
        const int32_t i = ord[r], mi = Q.seqmove[bk[i]];
        rs[r] = Q.src[mi];
        rd[r] = Q.dst[mi];
        rf[r] = bd[i];
    }
    gsync<G>();
    const long long we = Q.w[e];
    const int32_t lam = Q.PL.lam[e];
    for (int32_t r = gt; r < c; r += G) {
        const int32_t ps = rs[r], pd = rd[r];
        const int32_t fs = plist_find(Q.PL, a, lam, ps), fd = plist_find(Q.PL, a, lam, pd);
        int32_t cs = fs >= 0 ? Q.PL.cnt[fs] : 0, cd = fd >= 0 ? Q.PL.cnt[fd] : 0;
        int32_t is = fs >= 0 ? Q.PL.cin[fs] : 0, id = fd >= 0 ? Q.PL.cin[fd] : 0;
        for (int32_t t = 0; t < r; t++) {
            const int32_t xs = rs[t], xd = rd[t];
            const int32_t ds = (xd == ps) - (xs == ps), dd = (xd == pd) - (xs == pd);
            cs += ds;
            cd += dd;
            if (rf[t]) {
                is += ds;
                id += dd;
            }
        }
        const int32_t k = bk[ord[r]];
        long long g = 0;
        if (cs == 1) g += we;
        if (cd == 0) g -= we;
        if (g) atomicAdd(&Q.gseq[k], (unsigned long long)g);
        if (rf[r]) {
            if (is == 1) atomicAdd(&Q.dDs[k], -1);
            if (id == 0) atomicAdd(&Q.dDd[k], 1);
        }
    }
    gsync<G>();
}

// The hyperedges of `list` that hold a moved pin (lanes take one hyperedge
// each; those of more than 32 pins are scanned by the whole warp).
__global__ void k_touched(const int32_t *off, const int32_t *pin, const int32_t *mvpos, const int32_t *list,
                          int32_t count, int32_t *out, int32_t *out_n, int32_t *tout, int32_t *tout_n,
                          const int32_t *mcount) {
    HP_KERNEL_ENTER();
    if (*mcount == 0) return;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < count; base += step) {
        const int64_t i = base + lane;
        int32_t e = -1, a = 0, b = 0;
        if (i < count) {
            e = list[i];
            a = off[e];
            b = off[e + 1];
        }
        bool hit = false;
        if (e >= 0 && b - a <= 32)
            for (int32_t j = a; j < b && !hit; j++) hit = mvpos[pin[j]] >= 0;
        unsigned big = __ballot_sync(FULL, e >= 0 && b - a > 32);
        while (big) {
            const int l = __ffs(big) - 1;
            big &= big - 1;
            const int32_t ea = __shfl_sync(FULL, a, l), eb = __shfl_sync(FULL, b, l);
            bool found = false;
            for (int32_t j0 = ea; j0 < eb; j0 += 32) {
                const bool h = j0 + lane < eb && mvpos[pin[j0 + lane]] >= 0;
                if (__any_sync(FULL, h)) {
                    found = true;
                    break;
                }
            }
            if (lane == l) hit = found;
        }
        if (hit) {
            if (b - a <= TINY_E) tout[atomicAdd(tout_n, 1)] = e;
            else out[atomicAdd(out_n, 1)] = e;
        }
    }
}

constexpr int IS_T = 128;
// hyperedges of lo < |e| <= emax pins from the list, a warp each
__global__ void __launch_bounds__(IS_T) k_inseq_small(SeqSim Q, const int32_t *list, const int32_t *count_p,
                                                      int32_t emax, const int32_t *mcount, int32_t lo) {
    HP_KERNEL_ENTER();
    if (*mcount == 0) return;
    const int32_t count = *count_p;
    extern __shared__ __align__(16) int32_t sm[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int32_t *base = sm + wid * (9 * emax + 1);
    int32_t *bk = base, *bd = bk + emax, *ord = bd + emax, *tp = ord + emax, *tc = tp + 2 * emax,
            *tci = tc + 2 * emax, *gc = tci + 2 * emax;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < count; i += nw) {
        const int32_t e = list[i], sz = Q.off[e + 1] - Q.off[e];
        if (sz > lo && sz <= emax) inseq_edge<32>(Q, e, lane, bk, bd, ord, tp, tc, tci, gc);
    }
}
__global__ void __launch_bounds__(256) k_inseq_big(SeqSim Q, const int32_t *list, int32_t count, int32_t emax,
                                                   int32_t *gbuf, const int32_t *mcount) {
    HP_KERNEL_ENTER();
    if (*mcount == 0) return;
    __shared__ int32_t gc;
    int32_t *base = gbuf + (int64_t)blockIdx.x * 9 * (int64_t)emax;
    int32_t *bk = base, *bd = bk + emax, *ord = bd + emax, *tp = ord + emax, *tc = tp + 2 * emax,
            *tci = tc + 2 * emax;
    for (int32_t k = blockIdx.x; k < count; k += gridDim.x)
        inseq_edge<256>(Q, list[k], threadIdx.x, bk, bd, ord, tp, tc, tci, &gc);
}


// In-sequence gains of hyperedges of at most TINY_E pins, one thread each:
// the moved pins are taken in sequence order (ranks among at most TINY_E
// distinct positions) and the parts they leave or enter are tracked in a
// per-thread table of 2 TINY_E entries in shared memory.  The r-th moves of
// a warp's hyperedges are combined by sequence position (match_any) before
// their atomics: a moved node with many hyperedges is one position.
constexpr int IST_T = 128;
__global__ void __launch_bounds__(IST_T) k_inseq_tiny(SeqSim Q, const int32_t *list, const int32_t *count_p,
                                                       const int32_t *mcount) {
    HP_KERNEL_ENTER();
    __shared__ int32_t s_tab[IST_T * 6 * TINY_E];
    if (*mcount == 0) return;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const int32_t count = *count_p;
    int32_t *tp = s_tab + threadIdx.x * 6 * TINY_E, *tc = tp + 2 * TINY_E, *tci = tc + 2 * TINY_E;
    const int64_t step = (int64_t)gridDim.x * IST_T;
    for (int64_t base = blockIdx.x * (int64_t)IST_T + (threadIdx.x & ~31u); base < count; base += step) {
        const int64_t i = base + lane;
        int32_t a = 0, sz = 0, d0 = 0, lam = 0;
        long long we = 0;
        if (i < count) {
            const int32_t e = list[i];
            a = Q.off[e];
            sz = Q.off[e + 1] - a;
            d0 = Q.nsrc[e];
            we = Q.w[e];
            lam = Q.PL.lam[e];
        }
        int32_t kk[TINY_E];
        int nm = 0;
#pragma unroll
        for (int j = 0; j < TINY_E; j++) {
            kk[j] = 0x7fffffff;
            if (j < sz) {
                const int32_t k = Q.mvpos[Q.pin[a + j]];
                if (k >= 0) {
                    kk[j] = k;
                    nm++;
                }
            }
        }
        const int rmax = (int)__reduce_max_sync(FULL, (unsigned)nm);
        int nt = 0;
        for (int r = 0; r < rmax; r++) {
            int32_t k = -1;
            int g = 0, ds = 0, dd = 0;
            if (r < nm) {
                // the moved pin of rank r (positions are distinct)
                bool isdst = false;
#pragma unroll
                for (int j = 0; j < TINY_E; j++) {
                    int32_t rk = 0;
#pragma unroll
                    for (int x = 0; x < TINY_E; x++) rk += kk[x] < kk[j];
                    if (kk[j] != 0x7fffffff && rk == r) {
                        k = kk[j];
                        isdst = j >= d0;
                    }
                }
                const int32_t mi = Q.seqmove[k];
                const int32_t ps[2] = {Q.src[mi], Q.dst[mi]};
                int32_t sl[2];
                for (int h = 0; h < 2; h++) {
                    int32_t x = 0;
                    while (x < nt && tp[x] != ps[h]) x++;
                    if (x == nt) {
                        const int32_t f = plist_find(Q.PL, a, lam, ps[h]);
                        tp[x] = ps[h];
                        tc[x] = f >= 0 ? Q.PL.cnt[f] : 0;
                        tci[x] = f >= 0 ? Q.PL.cin[f] : 0;
                        nt++;
                    }
                    sl[h] = x;
                }
                if (tc[sl[0]] == 1) g += (int)we;
                if (tc[sl[1]] == 0) g -= (int)we;
                tc[sl[0]]--;
                tc[sl[1]]++;
                if (isdst) {
                    if (--tci[sl[0]] == 0) ds = -1;
                    if (++tci[sl[1]] == 1) dd = 1;
                }
            }
            // |g| <= 65536 per lane, so the warp sums fit 32 bits
            const unsigned grp = __match_any_sync(FULL, k);
            const int gs = (int)__reduce_add_sync(grp, (unsigned)g);
            const int dss = (int)__reduce_add_sync(grp, (unsigned)ds);
            const int dds = (int)__reduce_add_sync(grp, (unsigned)dd);
            if (k >= 0 && (grp & lt) == 0u) {
                if (gs) atomicAdd(&Q.gseq[k], (unsigned long long)(long long)gs);
                if (dss) atomicAdd(&Q.dDs[k], dss);
                if (dds) atomicAdd(&Q.dDd[k], dds);
            }
        }
    }
}

// ---------------------------------------------------------------- workspace
// Allocated once per call for the largest level and reused by every level
// and repetition.
struct LevelWs {
    // capacities
    int32_t cn, ce, nparts, cmax_e;
    int64_t cnp;
    // per level
    int32_t n, max_e, small_max, n_act, n_big;
    uint32_t pcap;
    int32_t *act, *big;
    long long *wns;
    int32_t *singin;
    Plist PL;
    RepArrays R;
    int32_t *cl, *hubs, *cw;
    int32_t *cflag, *cpos, *cut, *cut_off;   // cut incident hyperedges per node
    int32_t *tiny, n_tiny;                   // hyperedges of 2..8 pins
    int32_t *mid, n_mid;                     // hyperedges of 9..small_max pins
    int32_t parts_used;                      // parts holding a node at the level's start
    cudaStream_t side = nullptr;             // side stream of the hub gains
    cudaEvent_t ev[2] = {nullptr, nullptr};
    // algorithmic bytes of the repetitions (host): running total, and the cut
    // entries and their list entries of the last rebuilt repetition
    int64_t alg_bytes = 0, cuts = 0, cut_lam = 0;
    int32_t *touched, *ttouched;             // hyperedges with a moved pin (more than / at most 8 pins)
    Moves M, S;
    uint64_t *keys;
    uint32_t *idx;
    int32_t *msz, *mni;
    int32_t *first, *choice, *accnode, *pos, *clen, *lens, *starts, *cstart, *seqmove;
    unsigned long long *pen, *minpen, *acc1, *acc2;
    uint32_t *heads;
    uint64_t *hkeys;
    uint32_t *vkey, *vidx;
    long long *vsz;
    int32_t *vdd;
    long long *gsz, *gdd, *esz, *edd;
    int32_t *vhead;
    int32_t *ovf, *gk;
    long long *gc;
    uint32_t gcap;
    int gnb;
    int32_t *ptab, *ibuf;
    uint32_t bcap;
    int pnb;
    long long *bgain;
    int32_t *lvl;   // per-level counters
    int32_t *pmark; // [nparts] parts in use
};

static LevelWs *refine_workspace_body(LevelWs *W, int32_t n, int64_t np, int32_t e, int32_t nparts, int32_t max_e,
                                      const Params &P, Arena &A);

// on a failure half-way, the stream and events made so far are destroyed
// (the arena frees the device memory taken so far)
LevelWs *refine_workspace(int32_t n, int64_t np, int32_t e, int32_t nparts, int32_t max_e, const Params &P,
                          Arena &A) {
    LevelWs *W = new LevelWs();
    try {
        return refine_workspace_body(W, n, np, e, nparts, max_e, P, A);
    } catch (...) {
        if (W->side) cudaStreamDestroy(W->side);
        for (cudaEvent_t x : W->ev)
            if (x) cudaEventDestroy(x);
        delete W;
        throw;
    }
}

static LevelWs *refine_workspace_body(LevelWs *W, int32_t n, int64_t np, int32_t e, int32_t nparts, int32_t max_e,
                                      const Params &P, Arena &A) {
    cudaStream_t s = A.stream();
    HPC(cudaStreamCreateWithFlags(&W->side, cudaStreamNonBlocking));
    for (cudaEvent_t &x : W->ev) HPC(cudaEventCreateWithFlags(&x, cudaEventDisableTiming));
    W->cn = n;
    W->cnp = np;
    W->ce = e;
    W->nparts = nparts;
    W->cmax_e = max_e;
    W->act = A.get<int32_t>(e);
    W->big = A.get<int32_t>(e);
    W->wns = A.get<long long>(n);
    W->singin = A.get<int32_t>(n);
    W->PL.p = A.get<int32_t>(np);
    W->PL.cnt = A.get<int32_t>(np);
    W->PL.cin = A.get<int32_t>(np);
    W->PL.lam = A.get<int32_t>(e);
    RepArrays &R = W->R;
    R.nparts = nparts;
    R.rounds = P.o.chain_rounds;
    R.cnt = A.get<int32_t>(C_N);
    R.linked = A.get<int32_t>(P.o.chain_rounds + 1);
    R.D0 = A.get<int32_t>(nparts);
    R.psize = A.get<long long>(nparts);
    R.saving = A.get<long long>(n);
    R.pc = A.get<int32_t>(nparts + 1);
    R.pred = A.get<int32_t>(n);
    R.succ = A.get<int32_t>(n);
    R.chain = A.get<int32_t>(n);
    R.mvpos = A.get<int32_t>(n);
    R.cgain = A.get<long long>(n);
    R.gseq = A.get<unsigned long long>(n);
    R.acc0 = A.get<unsigned long long>(n);
    R.dDs = A.get<int32_t>(n);
    R.dDd = A.get<int32_t>(n);
    R.viol = A.get<int32_t>(n);
    W->cl = A.get<int32_t>(n);
    W->hubs = A.get<int32_t>(n);
    W->cw = A.get<int32_t>(n);
    W->cflag = A.get<int32_t>(np);
    W->cpos = A.get<int32_t>(np + 1);
    W->cut = A.get<int32_t>(np);
    W->cut_off = A.get<int32_t>(n + 1);
    W->tiny = A.get<int32_t>(e);
    W->mid = A.get<int32_t>(e);
    W->touched = A.get<int32_t>(e);
    W->ttouched = A.get<int32_t>(e);
    for (Moves *m : {&W->M, &W->S}) {
        m->node = A.get<int32_t>(n);
        m->src = A.get<int32_t>(n);
        m->dst = A.get<int32_t>(n);
        m->gain = A.get<long long>(n);
        m->count = R.cnt + C_MOVES;
    }
    W->keys = A.get<uint64_t>(n);
    W->idx = A.get<uint32_t>(n);
    W->msz = A.get<int32_t>(n);
    W->mni = A.get<int32_t>(n);
    W->first = A.get<int32_t>(nparts + 1);
    W->choice = A.get<int32_t>(n);
    W->accnode = A.get<int32_t>(n);
    W->pen = A.get<unsigned long long>(n);
    W->minpen = A.get<unsigned long long>(n);
    W->acc1 = A.get<unsigned long long>(n);
    W->acc2 = A.get<unsigned long long>(n);
    W->pos = A.get<int32_t>(n);
    W->clen = A.get<int32_t>(n);
    W->lens = A.get<int32_t>(n);
    W->starts = A.get<int32_t>(n);
    W->cstart = A.get<int32_t>(n);
    W->seqmove = A.get<int32_t>(n);
    W->heads = A.get<uint32_t>(n);
    W->hkeys = A.get<uint64_t>(n);
    W->vkey = A.get<uint32_t>(2 * (int64_t)n);
    W->vidx = A.get<uint32_t>(2 * (int64_t)n);
    W->vsz = A.get<long long>(2 * (int64_t)n);
    W->vdd = A.get<int32_t>(2 * (int64_t)n);
    W->gsz = A.get<long long>(2 * (int64_t)n);
    W->gdd = A.get<long long>(2 * (int64_t)n);
    W->esz = A.get<long long>(2 * (int64_t)n);
    W->edd = A.get<long long>(2 * (int64_t)n);
    W->vhead = A.get<int32_t>(std::max<int64_t>(nparts, 1));
    W->bgain = A.get<long long>(1);
    W->lvl = A.get<int32_t>(6);
    W->pmark = A.get<int32_t>(std::max(nparts, 1));
    // overflow tables of the gain kernel, one per CTA of its fallback grid
    W->gcap = pow2_at_least(2 * (int64_t)nparts + 2);
    W->gnb = (int)std::min<int64_t>(num_sms(), std::max<int64_t>(1, ((int64_t)1 << 27) / ((int64_t)W->gcap * 12)));
    W->ovf = A.get<int32_t>(n);
    W->gk = A.get<int32_t>((int64_t)W->gnb * 2 * W->gcap);
    W->gc = A.get<long long>((int64_t)W->gnb * W->gcap);
    fill_i32(W->gk, (int64_t)W->gnb * 2 * W->gcap, -1, s);
    HPC(cudaMemsetAsync(W->gc, 0, sizeof(long long) * W->gnb * W->gcap, s));
    // hyperedges above 512 pins: tables and buffers in global memory
    W->ptab = W->ibuf = nullptr;
    W->pnb = 0;
    if (max_e > 512) {
        W->bcap = pow2_at_least(2 * (int64_t)max_e);
        W->pnb = num_sms() * 2;
        W->ptab = A.get<int32_t>((int64_t)W->pnb * (3 * (int64_t)W->bcap + 4 * (int64_t)max_e));
        W->ibuf = A.get<int32_t>((int64_t)W->pnb * 9 * (int64_t)max_e);
    }
    return W;
}

void refine_workspace_free(LevelWs *W, Arena &A) {
    if (!W) return;
    // side-stream work must be done before the arena hands its memory back
    // (it is, unless the call is ending early on an error)
    if (W->side) {
        (void)cudaStreamSynchronize(W->side);
        cudaStreamDestroy(W->side);
    }
    for (cudaEvent_t x : W->ev)
        if (x) cudaEventDestroy(x);
    for (void *p : std::initializer_list<void *>{
             W->act, W->big, W->wns, W->singin, W->PL.p, W->PL.cnt, W->PL.cin, W->PL.lam, W->R.cnt, W->R.linked,
             W->R.D0, W->R.psize, W->R.saving, W->R.pc, W->R.pred, W->R.succ, W->R.chain, W->R.mvpos, W->R.cgain,
             W->R.gseq, W->R.acc0, W->R.dDs, W->R.dDd, W->R.viol, W->cl, W->hubs, W->cw, W->cflag, W->cpos, W->cut, W->cut_off, W->tiny, W->mid, W->touched, W->ttouched, W->M.node, W->M.src, W->M.dst, W->M.gain,
             W->S.node, W->S.src, W->S.dst, W->S.gain, W->keys, W->idx, W->msz, W->mni, W->first, W->choice, W->accnode, W->pen,
             W->minpen, W->acc1, W->acc2, W->pos, W->clen, W->lens, W->starts, W->cstart, W->seqmove, W->heads, W->hkeys,
             W->vkey, W->vidx, W->vsz, W->vdd, W->gsz, W->gdd, W->esz, W->edd, W->vhead, W->bgain, W->lvl, W->pmark, W->ovf, W->gk, W->gc, W->ptab, W->ibuf})
        A.release(p);
    delete W;
}

// per level: hyperedge classes and per-node constants
// parts holding at least one node (lambda(e) never exceeds it within a level:
// moves only go to parts that exist)
// the level's counters and per-part / per-node sums start at zero (one
// launch instead of four memsets, which would each end the overlap of a
// launch with its predecessor)
__global__ void k_prep_zero(int32_t *lvl, int32_t *pmark, int32_t nparts, long long *wns, int32_t *singin, int32_t n) {
    HP_KERNEL_ENTER();
    GRID_STRIDE(i, (int64_t)max(max(n, nparts), 6)) {
        if (i < 6) lvl[i] = 0;
        if (i < nparts) pmark[i] = 0;
        if (i < n) {
            wns[i] = 0;
            singin[i] = 0;
        }
    }
}

__global__ void k_used_parts(const int32_t *rho, int32_t n, int32_t *mark, int32_t *count) {
    HP_KERNEL_ENTER();
    GRID_STRIDE(v, (int64_t)n) {
        if (atomicExch(&mark[rho[v]], 1) == 0) atomicAdd(count, 1);
    }
}

static void level_prepare(const Level &L, const int32_t *w, const int32_t *rho, LevelWs &W, Arena &A) {
    cudaStream_t s = A.stream();
    const int32_t n = L.n, e = L.e;
    W.n = n;
    W.R.n = n;
    W.R.e = e;
    launch_k(k_prep_zero, grid_of(std::max(std::max(n, W.nparts), 6), 256), 256, 0, s, W.lvl, W.pmark, W.nparts, W.wns,
             W.singin, n);
    HP_LAUNCH_CHECK();
    if (e > 0) {
        launch_k(k_max_edge, grid_of(e, 256), 256, 0, s, L.off, e, W.lvl + 2);
        HP_LAUNCH_CHECK();
    }
    if (n > 0) {
        launch_k(k_used_parts, grid_of(n, 256), 256, 0, s, rho, n, W.pmark, W.lvl + 5);
        HP_LAUNCH_CHECK();
    }
    if (e > 0) {
        // the size classes take the largest hyperedge from the device (no read-back here)
        launch_k(k_level_edges, grid_of(e, 256), 256, 0, s, L.off, e, W.lvl + 2, W.act, W.big, W.tiny, W.mid, W.lvl);
        HP_LAUNCH_CHECK();
    }
    if (L.np > 0) {
        launch_k(k_level_nodes, grid_of(L.np, 256), 256, 0, s, L.off, L.ioff, L.inc, L.inode, L.nin, w, L.np, W.wns,
                 W.singin);
        HP_LAUNCH_CHECK();
    }
    int32_t hc[6];
    fetch_bytes(hc, W.lvl, sizeof hc, s);
    W.max_e = hc[2];
    W.small_max = level_small_max(W.max_e);
    W.n_act = hc[0];
    W.n_big = hc[1];
    W.n_tiny = hc[3];
    W.n_mid = hc[4];
    W.parts_used = hc[5];
    // pins lists of the level hold at most min(small_max, parts in use) entries
    W.pcap = pow2_at_least(2 * (int64_t)std::max<int32_t>(2, std::min<int32_t>(W.small_max, hc[5])));
    if (W.n_big > 0 && !W.ptab) throw Error(HP_ERR_INTERNAL, "large hyperedge buffers missing");
}

// One repetition; returns the number of moves applied.
// reuse: rho is unchanged since the previous repetition of this level (which
// applied nothing), so its pins lists, D(p), |p|, saving(v) and cut lists,
// all functions of rho, are reused instead of rebuilt
static int32_t rep_run(const Level &L, const int32_t *w, const Params &P, int32_t *rho, int second_half, LevelWs &W,
                       Arena &A, uint32_t *err_dev, const RepDebug *dbg, bool reuse = false) {
    cudaStream_t s = A.stream();
    const int32_t n = L.n, nparts = W.nparts;
    RepArrays &R = W.R;
    int32_t *cnt = R.cnt;
    const int64_t zspan = std::max<int64_t>(std::max<int64_t>(n, (int64_t)nparts + 1),
                                            std::max<int64_t>((int64_t)C_N, (int64_t)P.o.chain_rounds + 1));
    launch_k(k_rep_zero, grid_of(zspan, 256), 256, 0, s, R, reuse ? 1 : 0);
    HP_LAUNCH_CHECK();
    if (!reuse) {
        launch_k(k_rep_nodes, grid_of(n, 256), 256, 0, s, rho, L.size, W.singin, n, R.psize, R.D0);
        HP_LAUNCH_CHECK();
        // pins(p,e), pins_in(p,e), D(p), saving(v)
        if (W.n_mid > 0) {
            // hyperedges of up to MID_SPLIT pins in small tables (many warps
            // per SM), the rest of the warp tier in tables for small_max pins
            auto plist_mid = [&](uint32_t cap, int32_t lo, int32_t hi) {
                const int per = 5 * (int)cap + 1;
                size_t sm = (size_t)per * 4 * (PLW_T / 32);
                int occ = prepare_kernel((const void *)k_plist_small, PLW_T, sm);
                int grid = (int)std::min<int64_t>(cdiv(W.n_mid, PLW_T / 32), (int64_t)num_sms() * occ);
                launch_k(k_plist_small, std::max(grid, 1), PLW_T, sm, s, L.off, L.pin, L.nsrc, w, rho, W.n_mid, W.mid,
                         W.small_max, cap, W.PL, R.D0, R.saving, lo, hi);
                HP_LAUNCH_CHECK();
            };
            if (W.pcap > pow2_at_least(2 * MID_SPLIT)) {
                plist_mid(pow2_at_least(2 * MID_SPLIT), 0, MID_SPLIT);
                plist_mid(W.pcap, MID_SPLIT, INT32_MAX);
            } else {
                plist_mid(W.pcap, 0, INT32_MAX);
            }
        }
        if (W.n_tiny > 0) {
            launch_k(k_plist_tiny, grid_of(W.n_tiny, 128), 128, 0, s, L.off, L.pin, L.nsrc, w, rho, W.tiny, W.n_tiny, W.PL, R.D0,
                     R.saving);
            HP_LAUNCH_CHECK();
        }
        if (W.n_big > 0) {
            launch_k(k_plist_big, W.pnb, 256, 0, s, L.off, L.pin, L.nsrc, w, rho, W.big, W.n_big, W.bcap, W.ptab, W.cmax_e,
                     W.PL, R.D0, R.saving);
            HP_LAUNCH_CHECK();
        }
        // moves in isolation (Eq. 13)
        if (L.np > 0) {
            launch_k(k_cut_flags, grid_of(L.np, 256), 256, 0, s, L.off, L.pin, L.inc, L.inode, W.PL.lam, L.np, W.cflag,
                     reinterpret_cast<unsigned long long *>(cnt + C_ACC));
            HP_LAUNCH_CHECK();
        }
        scan_excl(W.cflag, W.cpos, L.np, W.cpos + L.np, A);
        launch_k(k_cut_fill, grid_of(std::max<int64_t>(L.np, (int64_t)n + 1), 256), 256, 0, s, L.inc, W.cflag, W.cpos, L.ioff,
                 L.np, n, W.cut, W.cut_off);
        HP_LAUNCH_CHECK();
    }
    launch_k(k_candidates, grid_of(n, 256), 256, 0, s, R.saving, W.cut_off, n, W.cl, cnt + C_CAND, W.hubs, cnt + C_HUB,
             W.cw, cnt + C_CW);
    HP_LAUNCH_CHECK();
    GainArgs G{L.off, W.cut_off, W.cut, w, rho, L.size, R.psize, R.saving, W.wns, W.PL, P.omega, second_half, W.M};
    uint32_t gcap_smem = 2048;
    if (P.o.debug_table_cap > 0) gcap_smem = (uint32_t)P.o.debug_table_cap;
    const size_t gsm = (size_t)gcap_smem * 12 + (size_t)(gcap_smem * 3 / 4) * 4;
    {
        // hub nodes on the side stream, beside the warp and CTA tiers (disjoint
        // node lists; all append to the same move and overflow lists by atomics)
        HPC(cudaEventRecord(W.ev[0], s));
        HPC(cudaStreamWaitEvent(W.side, W.ev[0], 0));
        const int occ_h = prepare_kernel((const void *)k_gains_smem<1024>, 1024, gsm);
        launch_k(k_gains_smem<1024>, num_sms() * std::max(occ_h, 1), 1024, gsm, W.side, G, W.hubs, cnt + C_HUB, gcap_smem,
                 W.ovf, cnt + C_OVF);
        HP_LAUNCH_CHECK();
        HPC(cudaEventRecord(W.ev[1], W.side));
    }
    {
        const uint32_t wlimit = P.o.debug_table_cap > 0 ? std::min<uint32_t>(GW_SLOTS * 3 / 4, P.o.debug_table_cap / 2)
                                                        : GW_SLOTS * 3 / 4;
        int occ = prepare_kernel((const void *)k_gains_warp, GW_T, 0);
        int grid = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, GW_T / 32), (int64_t)num_sms() * occ));
        launch_k(k_gains_warp, grid, GW_T, 0, s, G, W.cw, cnt + C_CW, wlimit, W.cl, cnt + C_CAND);
        HP_LAUNCH_CHECK();
    }
    {
        int occ = prepare_kernel((const void *)k_gains_smem<GN_T>, GN_T, gsm);
        int grid = std::max(1, std::min<int>(n, num_sms() * occ));
        launch_k(k_gains_smem<GN_T>, grid, GN_T, gsm, s, G, W.cl, cnt + C_CAND, gcap_smem, W.ovf, cnt + C_OVF);
        HP_LAUNCH_CHECK();
        HPC(cudaStreamWaitEvent(s, W.ev[1], 0));
        launch_k(k_gains_global, W.gnb, GN_T, 0, s, G, W.ovf, cnt + C_OVF, W.gcap, W.gk, W.gc, W.cl, cnt + C_BAD);
        HP_LAUNCH_CHECK();
    }
    // The rest of the repetition; `end` reads its counters back (the one
    // host read of a repetition on a small level) and returns the moves applied.
    auto end = [&]() -> int32_t {
        int32_t hc[C_N];
        fetch_bytes(hc, cnt, sizeof hc, s);
        if (hc[C_BAD]) throw Error(HP_ERR_INTERNAL, "gain table overflow");
        // algorithmic bytes (scope of Sec. VI-B..VI-D): a rebuilt repetition
        // reads each pin and its part (8 B) and writes the pins-list entries
        // (12 B each) and scans the incidence for cut hyperedges (4 B per
        // entry); every repetition reads the cut entries (4 B) and the list
        // entries behind them (12 B), and moves 48 B per proposed move (sort
        // read and write, sequence, in-sequence gain, two capacity events, apply)
        unsigned long long acc[3];
        std::memcpy(acc, hc + C_ACC, sizeof acc);
        if (!reuse) {
            W.alg_bytes += 12 * L.np + 12 * (int64_t)acc[0];
            W.cuts = (int64_t)acc[1];
            W.cut_lam = (int64_t)acc[2];
        }
        W.alg_bytes += 4 * W.cuts + 12 * W.cut_lam + 48 * (int64_t)hc[C_MOVES];
        return hc[C_APPLIED];
    };
    // Levels of at most SMALL_LEVEL nodes have at most that many moves, which
    // the cluster kernels sequence and validate whatever their number (none
    // included): no read-back is needed before the end of the repetition.
    const bool small_level = n <= SMALL_LEVEL && !dbg;
    int32_t m = n;   // an upper bound of the moves on small levels
    if (!small_level) {
        int32_t hc[C_N];
        fetch_bytes(hc, cnt, sizeof hc, s);
        if (hc[C_BAD]) throw Error(HP_ERR_INTERNAL, "gain table overflow");
        m = hc[C_MOVES];
        if (dbg) *dbg->m = m;
        if (m == 0) return end();
    }

    const long long gbound = std::max<long long>(P.wsum, 1);
    const int nb = bits_for((uint64_t)std::max(n - 1, 1)), gb = bits_for((uint64_t)gbound),
              sb = bits_for((uint64_t)std::max(nparts - 1, 1));
    const long long cgbound = (long long)std::min<double>((double)gbound * (double)std::max(n, 1), 9.0e18);
    const int cgb = bits_for((uint64_t)cgbound);
    const int packed = (10ll * P.omega + (long long)P.delta) < 0xffffffffll;
    ChainCtx C;
    C.window = P.o.chain_window;
    C.node = W.S.node;
    C.src = W.S.src;
    C.dst = W.S.dst;
    C.size = L.size;
    C.nin = L.nin;
    C.msz = W.msz;
    C.mni = W.mni;
    C.gain = W.S.gain;
    C.first = W.first;
    C.pred = R.pred;
    C.succ = R.succ;
    C.choice = W.choice;
    C.pen = W.pen;
    C.minpen = W.minpen;
    C.accnode = W.accnode;
    C.acc[0] = R.acc0;
    C.acc[1] = W.acc1;
    C.acc[2] = W.acc2;
    C.linked = R.linked;
    SeqCtx Q{W.S.node, R.pred, R.succ, W.S.gain, R.chain, W.pos, W.clen, R.cgain, err_dev};
    ValCtx V{W.seqmove, L.size, W.singin, R.dDs, R.dDd, R.D0, R.gseq, W.S, R.psize, W.vkey, W.vidx, W.vsz, W.vdd,
             R.viol, P.omega, P.delta, W.gsz, W.gdd, W.esz, W.edd, W.vhead};
    // one CTA sequences the moves unless the chaining window scans would be
    // long: every free end scans up to min(window, moves per part) moves of
    // its destination, each round (few parts in use make that quadratic)
    const int64_t per_part = cdiv(m, std::max<int32_t>(W.parts_used, 1));
    const int64_t scan_work = (int64_t)m * std::min<int64_t>(P.o.chain_window, per_part);
    // (on a larger level the device-wide path takes over above a few thousand
    // moves: the cluster's eight SMs then lose to the whole GPU's phases)
    const bool small = m <= SMALLM,
               one_cluster = small_level || (m <= SEQ_CLUSTER_M && scan_work <= (int64_t(1) << 21));
    if (one_cluster) {
        ClusterSeqArgs SA{W.M, W.S, W.keys, W.hkeys, W.idx, W.heads, W.first, W.lens, W.starts, W.cstart,
                          W.seqmove, R.mvpos, cnt, C, Q, nparts, P.o.chain_rounds, packed, gb, nb, sb, cgb, gbound,
                          cgbound};
        const size_t sm = SQ_SMEM;
        prepare_kernel((const void *)k_seq_cluster, SEQ_T, sm);
        launch_k(k_seq_cluster, SQ_CS, SEQ_T, sm, s, SA);
        HP_LAUNCH_CHECK();
    } else {
        // sort (p_s asc, gain desc, node asc)
        if (sb + gb + nb <= 64) {
            launch_k(k_move_keys, grid_of(m, 256), 256, 0, s, W.M, cnt + C_MOVES, gbound, gb, nb, -1, W.keys, W.idx, 1);
            HP_LAUNCH_CHECK();
            radix_sort_dev(W.keys, W.idx, cnt + C_MOVES, m, sb + gb + nb, A);
        } else {
            const int fb[3] = {nb, gb, sb};
            for (int f = 0; f < 3; f++) {
                launch_k(k_move_keys, grid_of(m, 256), 256, 0, s, W.M, cnt + C_MOVES, gbound, gb, nb, f, W.keys, W.idx,
                         f == 0);
                HP_LAUNCH_CHECK();
                radix_sort_dev(W.keys, W.idx, cnt + C_MOVES, m, fb[f], A);
            }
        }
        launch_k(k_gather_moves, grid_of(m, 256), 256, 0, s, W.M, W.idx, cnt + C_MOVES, W.S, R.pc, L.size, L.nin, W.msz,
                 W.mni);
        HP_LAUNCH_CHECK();
        scan_excl(R.pc, W.first, nparts + 1, nullptr, A);
        // chaining (Sec. VI-C)
        // (two passes per round here: on these levels the window scans are
        // long, and the one-pass round's extra slot read per scanned move
        // costs more than the barrier it saves)
        for (int32_t r = 0; r < P.o.chain_rounds; r++) {
            launch_k(k_choose, grid_of(m, 128), 128, 0, s, C, cnt + C_MOVES, r, packed);
            HP_LAUNCH_CHECK();
            if (!packed) {
                launch_k(k_accept_min, grid_of(m, 256), 256, 0, s, C, cnt + C_MOVES, r);
                HP_LAUNCH_CHECK();
                launch_k(k_accept_id, grid_of(m, 256), 256, 0, s, C, cnt + C_MOVES, r);
                HP_LAUNCH_CHECK();
            }
            launch_k(k_link, grid_of(m, 256), 256, 0, s, C, cnt + C_MOVES, r, packed);
            HP_LAUNCH_CHECK();
        }
        // chains in order of (total gain desc, head node asc)
        launch_k(k_path_heads, grid_of(m, 256), 256, 0, s, Q, cnt + C_MOVES);
        HP_LAUNCH_CHECK();
        launch_k(k_cycle_heads, grid_of(m, 256), 256, 0, s, Q, cnt + C_MOVES);
        HP_LAUNCH_CHECK();
        launch_k(k_head_collect, grid_of(m, 256), 256, 0, s, Q, cnt + C_MOVES, W.heads, cnt + C_NH);
        HP_LAUNCH_CHECK();
        if (cgb + nb <= 64) {
            launch_k(k_head_keys, grid_of(m, 256), 256, 0, s, W.heads, cnt + C_NH, R.cgain, W.S.node, cgbound, nb, -1,
                     W.hkeys);
            HP_LAUNCH_CHECK();
            radix_sort_dev(W.hkeys, W.heads, cnt + C_NH, m, cgb + nb, A);
        } else {
            for (int f = 0; f < 2; f++) {
                launch_k(k_head_keys, grid_of(m, 256), 256, 0, s, W.heads, cnt + C_NH, R.cgain, W.S.node, cgbound, nb, f,
                         W.hkeys);
                HP_LAUNCH_CHECK();
                radix_sort_dev(W.hkeys, W.heads, cnt + C_NH, m, f == 0 ? nb : cgb, A);
            }
        }
        launch_k(k_chain_lens, grid_of(m, 256), 256, 0, s, W.heads, cnt + C_NH, W.clen, m, W.lens);
        HP_LAUNCH_CHECK();
        scan_excl(W.lens, W.starts, m, nullptr, A);
        launch_k(k_chain_start, grid_of(m, 256), 256, 0, s, W.heads, cnt + C_NH, W.starts, W.cstart);
        HP_LAUNCH_CHECK();
        launch_k(k_seq_pos, grid_of(m, 256), 256, 0, s, R.chain, W.pos, W.cstart, cnt + C_MOVES, W.S.node, W.seqmove,
                 R.mvpos);
        HP_LAUNCH_CHECK();
    }
    if (dbg) {
        HPC(cudaMemcpyAsync(dbg->node, W.S.node, sizeof(int32_t) * m, cudaMemcpyDeviceToDevice, s));
        HPC(cudaMemcpyAsync(dbg->src, W.S.src, sizeof(int32_t) * m, cudaMemcpyDeviceToDevice, s));
        HPC(cudaMemcpyAsync(dbg->dst, W.S.dst, sizeof(int32_t) * m, cudaMemcpyDeviceToDevice, s));
        HPC(cudaMemcpyAsync(dbg->gain, W.S.gain, sizeof(long long) * m, cudaMemcpyDeviceToDevice, s));
        HPC(cudaMemcpyAsync(dbg->seq, W.seqmove, sizeof(int32_t) * m, cudaMemcpyDeviceToDevice, s));
    }

    // in-sequence gains and distinct-inbound changes per move
    SeqSim Z{L.off, L.pin, L.nsrc, w, R.mvpos, W.seqmove, W.S.src, W.S.dst, W.PL, R.gseq, R.dDs, R.dDd};
    if (W.n_act > 0) {
        launch_k(k_touched, grid_of(W.n_act, 256), 256, 0, s, L.off, L.pin, R.mvpos, W.act, W.n_act, W.touched,
                 cnt + C_TOUCH, W.ttouched, cnt + C_TTOUCH, cnt + C_MOVES);
        HP_LAUNCH_CHECK();
        launch_k(k_inseq_tiny, grid_of(W.n_act, IST_T), IST_T, 0, s, Z, W.ttouched, cnt + C_TTOUCH, cnt + C_MOVES);
        HP_LAUNCH_CHECK();
        auto inseq_mid = [&](int32_t lo, int32_t emax) {
            size_t sm = (size_t)(9 * emax + 1) * 4 * (IS_T / 32);
            int occ = prepare_kernel((const void *)k_inseq_small, IS_T, sm);
            int grid = (int)std::min<int64_t>(cdiv(W.n_act, IS_T / 32), (int64_t)num_sms() * occ);
            launch_k(k_inseq_small, std::max(grid, 1), IS_T, sm, s, Z, W.touched, cnt + C_TOUCH, emax, cnt + C_MOVES, lo);
            HP_LAUNCH_CHECK();
        };
        if (W.small_max > MID_SPLIT) {
            inseq_mid(0, MID_SPLIT);
            inseq_mid(MID_SPLIT, W.small_max);
        } else {
            inseq_mid(0, W.small_max);
        }
    }
    if (W.n_big > 0) {
        launch_k(k_inseq_big, W.pnb, 256, 0, s, Z, W.big, W.n_big, W.cmax_e, W.ibuf, cnt + C_MOVES);
        HP_LAUNCH_CHECK();
    }

    // validity of every prefix (Sec. VI-D), best valid prefix, apply
    if (small_level) {
        prepare_kernel((const void *)k_val_cluster, SQ_T, SQ_SMEM);
        launch_k(k_val_cluster, SQ_CS, SQ_T, SQ_SMEM, s, V, cnt, nparts, sb, W.bgain, rho);
        HP_LAUNCH_CHECK();
    } else if (small) {
        size_t sm = (size_t)2 * SMALLM * 2 * (4 + 4);
        prepare_kernel((const void *)k_val_small, SEQ_T, sm);
        launch_k(k_val_small, 1, SEQ_T, sm, s, V, cnt, nparts, sb, W.bgain, rho);
        HP_LAUNCH_CHECK();
    } else {
        launch_k(k_val_entries, grid_of(m, 256), 256, 0, s, V, cnt + C_MOVES, cnt + C_NV);
        HP_LAUNCH_CHECK();
        radix_sort_dev(W.vkey, W.vidx, cnt + C_NV, 2 * (int64_t)m, sb, A);
        launch_k(k_val_gather, grid_of(2 * (int64_t)m, 256), 256, 0, s, V, cnt + C_NV);
        HP_LAUNCH_CHECK();
        scan_excl((const int64_t *)W.gsz, (int64_t *)W.esz, 2 * (int64_t)m, nullptr, A);
        scan_excl((const int64_t *)W.gdd, (int64_t *)W.edd, 2 * (int64_t)m, nullptr, A);
        launch_k(k_val_trans, grid_of(2 * (int64_t)m, 256), 256, 0, s, V, cnt + C_NV);
        HP_LAUNCH_CHECK();
        launch_k(k_initial_bad, grid_of(nparts, 256), 256, 0, s, R.psize, R.D0, nparts, P.omega, P.delta, cnt + C_BAD0);
        HP_LAUNCH_CHECK();
        launch_k(k_best_prefix, 1, 1024, 0, s, R.gseq, R.viol, cnt + C_MOVES, cnt + C_BAD0, cnt + C_APPLIED, W.bgain);
        HP_LAUNCH_CHECK();
        launch_k(k_apply, grid_of(m, 256), 256, 0, s, W.seqmove, W.S.node, W.S.dst, cnt + C_APPLIED, rho);
        HP_LAUNCH_CHECK();
    }
    if (dbg) {
        HPC(cudaMemcpyAsync(dbg->gseq, R.gseq, sizeof(long long) * m, cudaMemcpyDeviceToDevice, s));
        HPC(cudaMemcpyAsync(dbg->best_gain, W.bgain, sizeof(long long), cudaMemcpyDeviceToDevice, s));
    }
    return end();
}

__global__ void k_max_edge_i(const int32_t *off, int32_t e, int32_t *maxe) {
    HP_KERNEL_ENTER();
    int32_t m = 0;
    GRID_STRIDE(i, (int64_t)e) m = max(m, off[i + 1] - off[i]);
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(maxe, m);
}

int32_t max_edge_size(const Level &L, Arena &A) {
    cudaStream_t s = A.stream();
    int32_t *mx = A.get<int32_t>(1);
    HPC(cudaMemsetAsync(mx, 0, sizeof(int32_t), s));
    if (L.e > 0) {
        launch_k(k_max_edge_i, grid_of(L.e, 256), 256, 0, s, L.off, L.e, mx);
        HP_LAUNCH_CHECK();
    }
    const int32_t r = fetch<int32_t>(mx, s);
    A.release(mx);
    return r;
}

int32_t refine_rep_debug(const Level &L, const int32_t *w, int32_t nparts, const Params &P, int32_t *rho,
                         int second_half, Arena &A, uint32_t *err_dev, const RepDebug &dbg) {
    *dbg.m = 0;
    if (L.n == 0) return 0;
    const int32_t max_e = max_edge_size(L, A);
    LevelWs *W = refine_workspace(L.n, L.np, L.e, nparts, max_e, P, A);
    level_prepare(L, w, rho, *W, A);
    int32_t k = rep_run(L, w, P, rho, second_half, *W, A, err_dev, &dbg);
    refine_workspace_free(W, A);
    return k;
}

RefineOut refine_level(const Level &L, const int32_t *w, const Params &P, int32_t *rho, LevelWs *W, Arena &A,
                       uint32_t *err_dev) {
    RefineOut out;
    if (L.n == 0 || P.o.theta == 0) return out;
    level_prepare(L, w, rho, *W, A);
    const int64_t bytes0 = W->alg_bytes;
    const int32_t half = P.o.theta / 2;
    bool same_rho = false;   // the previous repetition applied nothing
    for (int32_t rep = 0; rep < P.o.theta; rep++) {
        const int32_t k = rep_run(L, w, P, rho, rep >= half, *W, A, err_dev, nullptr, same_rho);
        same_rho = k == 0;
        out.reps++;
        out.moves += k;
        if (k == 0) {
            if (rep < half) rep = half - 1;
            else break;
        }
    }
    out.alg_bytes = W->alg_bytes - bytes0;
    return out;
}

// ---------------------------------------------------------------- final statistics
__global__ void k_part_sizes(const int32_t *part, int32_t n, long long *psize) {
    HP_KERNEL_ENTER();
    GRID_STRIDE(v, (int64_t)n) atomicAdd((unsigned long long *)&psize[part[v]], 1ull);
}
__global__ void k_part_max(const long long *psize, const int32_t *D, int32_t nparts, int32_t omega, int32_t delta,
                           long long *out) {
    HP_KERNEL_ENTER();
    long long ms = 0, md = 0, bad = 0;
    GRID_STRIDE(p, (int64_t)nparts) {
        ms = max(ms, psize[p]);
        md = max(md, (long long)D[p]);
        bad += (psize[p] > omega || D[p] > delta) ? 1 : 0;
    }
    for (int o = 16; o > 0; o >>= 1) {
        ms = max(ms, __shfl_down_sync(0xffffffffu, ms, o));
        md = max(md, __shfl_down_sync(0xffffffffu, md, o));
        bad += __shfl_down_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax((unsigned long long *)&out[2], (unsigned long long)ms);
        atomicMax((unsigned long long *)&out[3], (unsigned long long)md);
        atomicAdd((unsigned long long *)&out[4], (unsigned long long)bad);
    }
}

// out (device int64[5]): connectivity, cut-net, max part size, max distinct
// inbound hyperedges of a part, parts violating Omega or Delta
void part_stats(const Level &L, const int32_t *w, const int32_t *part, int32_t nparts, int32_t omega, int32_t delta,
                int64_t *out, Arena &A) {
    cudaStream_t s = A.stream();
    HPC(cudaMemsetAsync(out, 0, 5 * sizeof(int64_t), s));
    if (nparts <= 0) return;
    int32_t *D = A.get<int32_t>(nparts);
    long long *psize = A.get<long long>(nparts);
    HPC(cudaMemsetAsync(D, 0, sizeof(int32_t) * nparts, s));
    HPC(cudaMemsetAsync(psize, 0, sizeof(long long) * nparts, s));
    if (L.e > 0) {
        int32_t *maxe = A.get<int32_t>(1);
        HPC(cudaMemsetAsync(maxe, 0, sizeof(int32_t), s));
        launch_k(k_max_edge, grid_of(L.e, 256), 256, 0, s, L.off, L.e, maxe);
        HP_LAUNCH_CHECK();
        int32_t me = fetch<int32_t>(maxe, s);
        Plist PL;
        PL.p = A.get<int32_t>(L.np);
        PL.cnt = A.get<int32_t>(L.np);
        PL.cin = A.get<int32_t>(L.np);
        PL.lam = A.get<int32_t>(L.e);
        build_plist(L, w, part, me, PL, D, nullptr, A);
        launch_k(k_objective, grid_of(L.e, 256), 256, 0, s, PL.lam, w, L.e, (unsigned long long *)out,
                 (unsigned long long *)(out + 1));
        HP_LAUNCH_CHECK();
        A.release(PL.p);
        A.release(PL.cnt);
        A.release(PL.cin);
        A.release(PL.lam);
        A.release(maxe);
    }
    launch_k(k_part_sizes, grid_of(L.n, 256), 256, 0, s, part, L.n, psize);
    HP_LAUNCH_CHECK();
    launch_k(k_part_max, grid_of(nparts, 256), 256, 0, s, psize, D, nparts, omega, delta, (long long *)out);
    HP_LAUNCH_CHECK();
    A.release(D);
    A.release(psize);
}

}  // namespace hp
