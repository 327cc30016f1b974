// hp_refine.cu -- one level of refinement (Sec. VI): Theta repetitions of
//   pins(p,e) lists  -> move proposal by gain (Eq. 13, Sec. VI-B)
//   -> sort (p_s asc, gain desc, node asc) -> chaining (Sec. VI-C)
//   -> chain order -> in-sequence gains (Eq. 14-15, exact change of
//   connectivity) -> event-based validity of every prefix (Sec. VI-D)
//   -> apply the best valid prefix.
// pins(p,e) is kept as a short list per hyperedge, sorted by partition id, at
// the hyperedge's own pin segment: (p, pins(p,e), pins_in(p,e)).
#include <cuda_runtime.h>

#include <algorithm>

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

__device__ __forceinline__ uint32_t hslot(int32_t x, uint32_t mask) { return ((uint32_t)x * 0x9E3779B1u) & mask; }

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

// edges with |e| <= small_max, one warp each, tables in shared memory
__global__ void __launch_bounds__(PLW_T) k_plist_small(const int32_t *off, const int32_t *pin, const int32_t *nsrc,
                                                       const int32_t *w, const int32_t *rho, int32_t e,
                                                       int32_t small_max, uint32_t cap, Plist PL, int32_t *D,
                                                       long long *saving) {
    extern __shared__ __align__(16) int32_t sm[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int per = 3 * (int)cap + 4 * small_max + 1;
    int32_t *base = sm + wid * per;
    int32_t *keys = base, *tc = base + cap, *tci = base + 2 * cap;
    int32_t *es = base + 3 * cap, *ep = es + small_max, *ec = ep + small_max, *eci = ec + small_max,
            *gcnt = eci + small_max;
    for (uint32_t i = lane; i < cap; i += 32) {
        keys[i] = -1;
        tc[i] = 0;
        tci[i] = 0;
    }
    __syncwarp();
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < e; i += nw) {
        if (off[i + 1] - off[i] > small_max) continue;
        plist_edge<32>((int32_t)i, lane, off, pin, nsrc, w, rho, keys, tc, tci, cap, es, ep, ec, eci, gcnt, PL, D,
                       saving);
    }
}

// edges with |e| > small_max, one CTA each, tables in global memory
__global__ void __launch_bounds__(256) k_plist_big(const int32_t *off, const int32_t *pin, const int32_t *nsrc,
                                                   const int32_t *w, const int32_t *rho, const int32_t *list,
                                                   int32_t count, uint32_t cap, int32_t *gtab, int32_t max_e, Plist PL,
                                                   int32_t *D, long long *saving) {
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
    GRID_STRIDE(i, (int64_t)e) {
        int32_t sz = off[i + 1] - off[i];
        if (sz > small_max) {
            list[atomicAdd(cnt, 1)] = (int32_t)i;
            atomicMax(maxe, sz);
        }
    }
}

__global__ void k_max_edge(const int32_t *off, int32_t e, int32_t *maxe) {
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
    const int per = 3 * (int)cap + 4 * small_max + 1;
    size_t sm = (size_t)per * 4 * (PLW_T / 32);
    HPC(cudaFuncSetAttribute(k_plist_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int occ = 0;
    HPC(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_plist_small, PLW_T, sm));
    int grid = (int)std::min<int64_t>(cdiv(L.e, PLW_T / 32), (int64_t)num_sms() * std::max(occ, 1));
    k_plist_small<<<std::max(grid, 1), PLW_T, sm, s>>>(L.off, L.pin, L.nsrc, w, rho, L.e, small_max, cap, PL, D,
                                                       saving);
    HP_LAUNCH_CHECK();
    if (max_e > small_max) {
        int32_t *list = A.get<int32_t>(L.e);
        int32_t *cnt = A.get<int32_t>(2);
        HPC(cudaMemsetAsync(cnt, 0, 2 * sizeof(int32_t), s));
        k_big_edges<<<grid_of(L.e, 256), 256, 0, s>>>(L.off, L.e, small_max, list, cnt, cnt + 1);
        HP_LAUNCH_CHECK();
        int32_t hc[2];
        fetch_bytes(hc, cnt, sizeof hc, s);
        if (hc[0] > 0) {
            uint32_t bcap = pow2_at_least(2 * (int64_t)hc[1]);
            int nb = std::min<int>(hc[0], num_sms() * 2);
            int32_t *gtab = A.get<int32_t>((int64_t)nb * (3 * (int64_t)bcap + 4 * (int64_t)hc[1]));
            k_plist_big<<<nb, 256, 0, s>>>(L.off, L.pin, L.nsrc, w, rho, list, hc[0], bcap, gtab, hc[1], PL, D,
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
    k_max_edge<<<grid_of(L.e, 256), 256, 0, s>>>(L.off, L.e, maxe);
    HP_LAUNCH_CHECK();
    int32_t me = fetch<int32_t>(maxe, s);
    Plist PL;
    PL.p = A.get<int32_t>(L.np);
    PL.cnt = A.get<int32_t>(L.np);
    PL.cin = A.get<int32_t>(L.np);
    PL.lam = A.get<int32_t>(L.e);
    build_plist(L, w, rho, me, PL, nullptr, nullptr, A);
    k_objective<<<grid_of(L.e, 256), 256, 0, s>>>(PL.lam, w, L.e, (unsigned long long *)conn_dev,
                                                  (unsigned long long *)cutnet_dev);
    HP_LAUNCH_CHECK();
    A.release(PL.p);
    A.release(PL.cnt);
    A.release(PL.cin);
    A.release(PL.lam);
    A.release(maxe);
}

// ---------------------------------------------------------------- per level constants
// Wns(v) = sum of w(e) over incident hyperedges with |e| >= 2
__global__ void k_wns(const int32_t *off, const int32_t *ioff, const int32_t *inc, const int32_t *w, int32_t n,
                      long long *wns) {
    GRID_STRIDE(v, (int64_t)n) {
        long long s = 0;
        for (int32_t t = ioff[v]; t < ioff[v + 1]; t++) {
            int32_t e = inc[t];
            if (off[e + 1] - off[e] >= 2) s += w[e];
        }
        wns[v] = s;
    }
}

__global__ void k_psize(const int32_t *rho, const int32_t *size, int32_t n, long long *psize) {
    GRID_STRIDE(v, (int64_t)n) atomicAdd((unsigned long long *)&psize[rho[v]], (unsigned long long)size[v]);
}

__global__ void k_candidates(const long long *saving, int32_t n, int32_t *list, int32_t *cnt) {
    GRID_STRIDE(v, (int64_t)n) {
        if (saving[v] > 0) list[atomicAdd(cnt, 1)] = (int32_t)v;
    }
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
                           long long *conn, uint32_t cap, uint32_t limit, int32_t *s_cnt, int *s_flag, Moves M,
                           int32_t *ovf, int32_t *ovf_n, long long *s_rg, int32_t *s_rp) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t mask = cap - 1;
    const int32_t s = rho[v];
    for (int32_t t = ioff[v] + wid; t < ioff[v + 1]; t += nw) {
        if (*(volatile int *)s_flag) break;
        int32_t e = inc[t];
        int32_t a = off[e];
        if (off[e + 1] - a < 2) continue;
        const long long we = w[e];
        const int32_t lam = PL.lam[e];
        for (int32_t k = lane; k < lam; k += 32) {
            int32_t p = PL.p[a + k];
            if (p == s) continue;
            uint32_t h = hslot(p, mask);
            for (uint32_t probe = 0; probe < cap; probe++) {
                int32_t kk = ((volatile int32_t *)keys)[h];
                if (kk == -1) {
                    int32_t old = atomicCAS(&keys[h], -1, p);
                    if (old == -1) {
                        if ((uint32_t)atomicAdd(s_cnt, 1) + 1 > limit) *(volatile int *)s_flag = 1;
                        kk = p;
                    } else {
                        kk = old;
                    }
                }
                if (kk == p) {
                    atomicAdd((unsigned long long *)&conn[h], (unsigned long long)we);
                    break;
                }
                h = (h + 1) & mask;
            }
        }
    }
    __syncthreads();
    const int overflow = *s_flag;
    long long bg = 0;
    int32_t bp = -1;
    const long long base = saving[v] - wns[v];
    for (uint32_t h = threadIdx.x; h < cap; h += blockDim.x) {
        int32_t p = keys[h];
        if (p >= 0) {
            if (!overflow && (!second_half || (long long)size[v] + psize[p] <= omega)) {
                long long g = base + conn[h];
                if (bp < 0 || g > bg || (g == bg && p > bp)) {
                    bg = g;
                    bp = p;
                }
            }
            keys[h] = -1;
            conn[h] = 0;
        }
    }
    if (overflow) {
        __syncthreads();
        if (threadIdx.x == 0) {
            ovf[atomicAdd(ovf_n, 1)] = v;
            *s_flag = 0;
            *s_cnt = 0;
        }
        __syncthreads();
        return;
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

__global__ void __launch_bounds__(GN_T) k_gains_smem(GainArgs G, const int32_t *list, int32_t count, uint32_t cap,
                                                     int32_t *ovf, int32_t *ovf_n) {
    extern __shared__ __align__(16) unsigned char smem[];
    long long *conn = reinterpret_cast<long long *>(smem);
    int32_t *keys = reinterpret_cast<int32_t *>(conn + cap);
    __shared__ int32_t s_cnt;
    __shared__ int s_flag;
    __shared__ long long s_rg[8];
    __shared__ int32_t s_rp[8];
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
                   G.second_half, keys, conn, cap, cap * 3 / 4, &s_cnt, &s_flag, G.M, ovf, ovf_n, s_rg, s_rp);
}

__global__ void __launch_bounds__(GN_T) k_gains_global(GainArgs G, const int32_t *list, int32_t count, uint32_t cap,
                                                       int32_t *gkeys, long long *gconn, int32_t *bad,
                                                       int32_t *bad_n) {
    __shared__ int32_t s_cnt;
    __shared__ int s_flag;
    __shared__ long long s_rg[8];
    __shared__ int32_t s_rp[8];
    int32_t *keys = gkeys + (int64_t)blockIdx.x * cap;
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
                   G.second_half, keys, conn, cap, cap - 1, &s_cnt, &s_flag, G.M, bad, bad_n, s_rg, s_rp);
}

// ---------------------------------------------------------------- sort of moves
__global__ void k_move_keys(const Moves M, const int32_t *cntp, long long gmax, int gb, int nb, uint64_t *keys,
                            uint32_t *idx) {
    int32_t m = *cntp;
    GRID_STRIDE(i, (int64_t)m) {
        uint64_t k = ((uint64_t)M.src[i] << (gb + nb)) | ((uint64_t)(gmax - M.gain[i]) << nb) | (uint64_t)M.node[i];
        keys[i] = k;
        idx[i] = (uint32_t)i;
    }
}
__global__ void k_gather_moves(const Moves M, const uint32_t *idx, int32_t m, Moves S) {
    GRID_STRIDE(i, (int64_t)m) {
        uint32_t k = idx[i];
        S.node[i] = M.node[k];
        S.src[i] = M.src[k];
        S.dst[i] = M.dst[k];
        S.gain[i] = M.gain[k];
    }
}
__global__ void k_max_gain(const long long *gain, int32_t m, unsigned long long *gmax) {
    unsigned long long g = 0;
    GRID_STRIDE(i, (int64_t)m) g = max(g, (unsigned long long)gain[i]);
    for (int o = 16; o > 0; o >>= 1) g = max(g, __shfl_down_sync(0xffffffffu, g, o));
    if ((threadIdx.x & 31) == 0) atomicMax(gmax, g);
}
// generic path: keys of one field at a time (stable LSD over three sorts)
__global__ void k_field_keys(const Moves M, int32_t m, int field, long long gmax, uint64_t *keys, const uint32_t *idx) {
    GRID_STRIDE(i, (int64_t)m) {
        uint32_t k = idx[i];
        keys[i] = field == 0 ? (uint64_t)M.node[k] : field == 1 ? (uint64_t)(gmax - M.gain[k]) : (uint64_t)M.src[k];
    }
}

// ---------------------------------------------------------------- chaining
__global__ void k_part_count(const int32_t *src, int32_t m, int32_t *cnt) {
    GRID_STRIDE(i, (int64_t)m) atomicAdd(&cnt[src[i]], 1);
}

struct ChainCtx {
    int32_t m, window;
    const int32_t *node, *src, *dst, *size, *nin;
    const long long *gain;
    const int32_t *first;   // [nparts+1]
    int32_t *pred, *succ, *choice;
    unsigned long long *pen, *minpen;
    int32_t *accnode;
    int32_t *linked;
};

// every free chain end picks, among the first `window` moves leaving its
// destination that have no predecessor, the one of maximum grade
// G = gain(m)*10^7 - 10|size(n)-size(m)| - |nin(n)-nin(m)|, earliest on ties.
__global__ void k_choose(ChainCtx C) {
    GRID_STRIDE(i0, (int64_t)C.m) {
        int32_t i = (int32_t)i0;
        C.choice[i] = -1;
        if (C.succ[i] >= 0) continue;
        int32_t d = C.dst[i];
        int32_t seen = 0, best = -1;
        __int128 bG = 0;
        unsigned long long bpen = 0;
        const int32_t vi = C.node[i];
        for (int32_t j = C.first[d]; j < C.first[d + 1] && seen < C.window; j++) {
            if (C.pred[j] >= 0 || j == i) continue;
            seen++;
            int32_t vj = C.node[j];
            long long ds = (long long)C.size[vi] - C.size[vj];
            long long di = (long long)C.nin[vi] - C.nin[vj];
            unsigned long long pen = 10ull * (unsigned long long)(ds < 0 ? -ds : ds) + (unsigned long long)(di < 0 ? -di : di);
            __int128 G = (__int128)C.gain[j] * 10000000 - (__int128)pen;
            if (best < 0 || G > bG) {
                best = j;
                bG = G;
                bpen = pen;
            }
        }
        C.choice[i] = best;
        C.pen[i] = bpen;
    }
}
// for a chosen move, choosers compare by G; G differs only by the penalty
__global__ void k_accept_min(ChainCtx C) {
    GRID_STRIDE(i, (int64_t)C.m) {
        int32_t j = C.choice[i];
        if (j >= 0) atomicMin(&C.minpen[j], C.pen[i]);
    }
}
__global__ void k_accept_id(ChainCtx C) {
    GRID_STRIDE(i, (int64_t)C.m) {
        int32_t j = C.choice[i];
        if (j >= 0 && C.pen[i] == C.minpen[j]) atomicMax(&C.accnode[j], C.node[i]);
    }
}
__global__ void k_link(ChainCtx C) {
    GRID_STRIDE(i, (int64_t)C.m) {
        int32_t j = C.choice[i];
        if (j >= 0 && C.pen[i] == C.minpen[j] && C.accnode[j] == C.node[i]) {
            C.pred[j] = (int32_t)i;
            C.succ[i] = j;
            *C.linked = 1;
        }
    }
}

// ---------------------------------------------------------------- chain order
struct SeqCtx {
    int32_t m;
    const int32_t *node, *pred, *succ;
    const long long *gain;
    int32_t *chain, *pos, *clen;
    long long *cgain;
    uint32_t *err;
};
__global__ void k_path_heads(SeqCtx S) {
    GRID_STRIDE(i0, (int64_t)S.m) {
        int32_t i = (int32_t)i0;
        if (S.pred[i] >= 0) continue;
        long long g = 0;
        int32_t k = 0;
        for (int32_t j = i; j >= 0; j = S.succ[j]) {
            if (k > S.m) {
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
__global__ void k_cycle_heads(SeqCtx S) {
    GRID_STRIDE(i0, (int64_t)S.m) {
        int32_t i = (int32_t)i0;
        if (S.chain[i] >= 0) continue;
        int32_t mn = S.node[i], k = 0;
        for (int32_t j = S.succ[i]; j != i; j = S.succ[j]) {
            if (j < 0 || ++k > S.m) {
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
        } while (j != i && c <= S.m);
        S.clen[i] = c;
        S.cgain[i] = g;
    }
}
__global__ void k_head_flags(const int32_t *chain, int32_t m, int32_t *flag) {
    GRID_STRIDE(i, (int64_t)m) flag[i] = chain[i] == (int32_t)i ? 1 : 0;
}
__global__ void k_head_compact(const int32_t *flag, const int32_t *pos, int32_t m, uint32_t *heads) {
    GRID_STRIDE(i, (int64_t)m) {
        if (flag[i]) heads[pos[i]] = (uint32_t)i;
    }
}
__global__ void k_head_keys(const uint32_t *heads, int32_t nh, const long long *cgain, const int32_t *node,
                            long long gmax, int nb, int field, uint64_t *keys) {
    GRID_STRIDE(k, (int64_t)nh) {
        uint32_t h = heads[k];
        uint64_t gk = (uint64_t)(gmax - cgain[h]);
        if (field < 0) keys[k] = (gk << nb) | (uint64_t)node[h];
        else keys[k] = field == 0 ? (uint64_t)node[h] : gk;
    }
}
__global__ void k_chain_lens(const uint32_t *heads, int32_t nh, const int32_t *clen, int32_t *lens) {
    GRID_STRIDE(k, (int64_t)nh) lens[k] = clen[heads[k]];
}
__global__ void k_chain_start(const uint32_t *heads, int32_t nh, const int32_t *starts, int32_t *cstart) {
    GRID_STRIDE(k, (int64_t)nh) cstart[heads[k]] = starts[k];
}
__global__ void k_seq_pos(const int32_t *chain, const int32_t *pos, const int32_t *cstart, int32_t m, int32_t *seqpos,
                          int32_t *seqmove) {
    GRID_STRIDE(i, (int64_t)m) {
        int32_t k = cstart[chain[i]] + pos[i];
        seqpos[i] = k;
        seqmove[k] = (int32_t)i;
    }
}

// ---------------------------------------------------------------- in-sequence gains
// Events of move k (node v: s -> d) on every e in I(v): (e, s, k, -1) and
// (e, d, k, +1).  Sorted by (e, p, k), each (e, p) run is walked with the
// running pins(p,e) and pins_in(p,e): a -1 event that empties e in p spares
// w(e), a +1 event that enters an empty p costs w(e) (Eq. 14-15 read as the
// exact change of connectivity); inbound 1->0 and 0->1 transitions give the
// distinct-inbound events of Sec. VI-D.
__global__ void k_ev_count(const int32_t *seqmove, const int32_t *node, const int32_t *ioff, int32_t m,
                           int32_t *cnt) {
    GRID_STRIDE(k, (int64_t)m) {
        int32_t v = node[seqmove[k]];
        cnt[k] = 2 * (ioff[v + 1] - ioff[v]);
    }
}
struct EvCtx {
    int32_t m, e_bits, p_bits, k_bits;
    const int32_t *seqmove, *node, *src, *dst, *ioff, *inc, *nin;
    const int32_t *evoff;
    uint64_t *keys;
    uint32_t *vals;   // bit 0: +1 event, bit 1: inbound (v is a destination of e)
};
__global__ void k_ev_gen(EvCtx E) {
    GRID_STRIDE(k, (int64_t)E.m) {
        int32_t i = E.seqmove[k];
        int32_t v = E.node[i], s = E.src[i], d = E.dst[i];
        int32_t o = E.evoff[k];
        int32_t a = E.ioff[v], b = E.ioff[v + 1], mi = a + E.nin[v];
        for (int32_t t = a; t < b; t++) {
            uint64_t e = (uint64_t)E.inc[t];
            uint32_t inb = t < mi ? 2u : 0u;
            E.keys[o] = (((e << E.p_bits) | (uint64_t)s) << E.k_bits) | (uint64_t)k;
            E.vals[o] = inb;
            o++;
            E.keys[o] = (((e << E.p_bits) | (uint64_t)d) << E.k_bits) | (uint64_t)k;
            E.vals[o] = inb | 1u;
            o++;
        }
    }
}

__device__ __forceinline__ int32_t plist_find(const Plist &PL, int32_t a, int32_t lam, int32_t p) {
    int32_t lo = 0, hi = lam;
    while (lo < hi) {
        int32_t mid = (lo + hi) >> 1;
        if (PL.p[a + mid] < p) lo = mid + 1;
        else hi = mid;
    }
    return (lo < lam && PL.p[a + lo] == p) ? a + lo : -1;
}

struct WalkCtx {
    int64_t nev;
    int32_t p_bits, k_bits;
    const uint64_t *keys;
    const uint32_t *vals;
    const int32_t *off, *w;
    Plist PL;
    unsigned long long *gseq;   // [m] (two's complement sums)
    uint64_t *dkeys;            // distinct-inbound events: key (p, k)
    int32_t *dvals;             // +1 / -1
    int32_t *dcount;
};
__global__ void k_ev_walk(WalkCtx W) {
    const uint64_t kmask = (1ull << W.k_bits) - 1, pmask = (1ull << W.p_bits) - 1;
    GRID_STRIDE(i, W.nev) {
        uint64_t key = W.keys[i];
        uint64_t ep = key >> W.k_bits;
        if (i > 0 && (W.keys[i - 1] >> W.k_bits) == ep) continue;   // not the head of its (e, p) run
        int32_t e = (int32_t)(ep >> W.p_bits), p = (int32_t)(ep & pmask);
        int32_t a = W.off[e];
        int32_t f = plist_find(W.PL, a, W.PL.lam[e], p);
        int32_t c = f >= 0 ? W.PL.cnt[f] : 0, ci = f >= 0 ? W.PL.cin[f] : 0;
        const long long we = W.w[e];
        for (int64_t j = i; j < W.nev && (W.keys[j] >> W.k_bits) == ep; j++) {
            int32_t k = (int32_t)(W.keys[j] & kmask);
            uint32_t val = W.vals[j];
            bool plus = val & 1u, inb = val & 2u;
            if (plus) {
                if (c == 0) atomicAdd(&W.gseq[k], (unsigned long long)(-we));
                c++;
                if (inb) {
                    if (ci == 0) {
                        int32_t o = atomicAdd(W.dcount, 1);
                        W.dkeys[o] = ((uint64_t)p << W.k_bits) | (uint64_t)k;
                        W.dvals[o] = 1;
                    }
                    ci++;
                }
            } else {
                if (c == 1) atomicAdd(&W.gseq[k], (unsigned long long)we);
                c--;
                if (inb) {
                    ci--;
                    if (ci == 0) {
                        int32_t o = atomicAdd(W.dcount, 1);
                        W.dkeys[o] = ((uint64_t)p << W.k_bits) | (uint64_t)k;
                        W.dvals[o] = -1;
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------------- validity
// All capacity events of the sequence, keyed (p, k): size events (-size at
// p_s, +size at p_d) and distinct-inbound events.  Per part, walk them in
// sequence order and record every change of the part's validity at k.
struct ValCtx {
    int64_t nev;
    int32_t k_bits;
    const uint64_t *keys;
    const uint32_t *idx;       // index into the payload arrays
    const long long *dsize;
    const int32_t *dd;
    const long long *psize;
    const int32_t *D0;
    int32_t omega, delta;
    int32_t *viol;             // [m] change of the number of invalid parts at k
};
__global__ void k_size_events(const int32_t *seqmove, const int32_t *node, const int32_t *src, const int32_t *dst,
                              const int32_t *size, int32_t m, int32_t k_bits, uint64_t *keys, long long *dsize,
                              int32_t *dd, int64_t base) {
    GRID_STRIDE(k, (int64_t)m) {
        int32_t i = seqmove[k];
        long long sz = size[node[i]];
        keys[base + 2 * k] = ((uint64_t)src[i] << k_bits) | (uint64_t)k;
        dsize[base + 2 * k] = -sz;
        dd[base + 2 * k] = 0;
        keys[base + 2 * k + 1] = ((uint64_t)dst[i] << k_bits) | (uint64_t)k;
        dsize[base + 2 * k + 1] = sz;
        dd[base + 2 * k + 1] = 0;
    }
}
__global__ void k_d_events(const uint64_t *dkeys, const int32_t *dvals, int32_t nd, uint64_t *keys, long long *dsize,
                           int32_t *dd) {
    GRID_STRIDE(i, (int64_t)nd) {
        keys[i] = dkeys[i];
        dsize[i] = 0;
        dd[i] = dvals[i];
    }
}
__global__ void k_val_walk(ValCtx V) {
    const uint64_t kmask = (1ull << V.k_bits) - 1;
    GRID_STRIDE(i, V.nev) {
        uint64_t key = V.keys[i];
        uint64_t p64 = key >> V.k_bits;
        if (i > 0 && (V.keys[i - 1] >> V.k_bits) == p64) continue;
        int32_t p = (int32_t)p64;
        long long sz = V.psize[p];
        long long dcnt = V.D0[p];
        bool valid = sz <= V.omega && dcnt <= V.delta;
        int64_t j = i;
        while (j < V.nev && (V.keys[j] >> V.k_bits) == p64) {
            uint64_t kk = V.keys[j] & kmask;
            while (j < V.nev && V.keys[j] == ((p64 << V.k_bits) | kk)) {
                uint32_t x = V.idx[j];
                sz += V.dsize[x];
                dcnt += V.dd[x];
                j++;
            }
            bool nv = sz <= V.omega && dcnt <= V.delta;
            if (nv != valid) atomicAdd(&V.viol[kk], nv ? -1 : 1);
            valid = nv;
        }
    }
}
__global__ void k_initial_bad(const long long *psize, const int32_t *D0, int32_t nparts, int32_t omega, int32_t delta,
                              int32_t *bad) {
    int32_t c = 0;
    GRID_STRIDE(p, (int64_t)nparts) c += (psize[p] > omega || D0[p] > delta) ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(bad, c);
}

// best prefix: max cumulative gain with zero invalid parts, longest on ties
__global__ void __launch_bounds__(1024) k_best_prefix(const unsigned long long *gseq, const int32_t *violc, int32_t m,
                                                      const int32_t *bad0, int32_t *best_len, long long *best_gain) {
    __shared__ long long s_g[32];
    __shared__ int32_t s_k[32];
    __shared__ long long s_carry_g;
    __shared__ int32_t s_carry_v;
    if (threadIdx.x == 0) {
        s_carry_g = 0;
        s_carry_v = *bad0;
    }
    __syncthreads();
    long long bestg = 0;
    int32_t bestk = 0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int32_t base = 0; base < m; base += 1024) {
        int32_t k = base + threadIdx.x;
        long long g = k < m ? (long long)gseq[k] : 0;
        int32_t dv = k < m ? violc[k] : 0;
        // block inclusive scans of g and dv
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
    // reduce (bestg, bestk): larger gain, then larger k
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
}

__global__ void k_apply(const int32_t *seqmove, const int32_t *node, const int32_t *dst, const int32_t *lenp,
                        int32_t *rho) {
    int32_t L = *lenp;
    GRID_STRIDE(k, (int64_t)L) {
        int32_t i = seqmove[k];
        rho[node[i]] = dst[i];
    }
}

// ---------------------------------------------------------------- one repetition
static int32_t refine_rep(const Level &L, const int32_t *w, int32_t nparts, const Params &P, int32_t *rho,
                          int second_half, int32_t max_e, const long long *wns, Arena &A, uint32_t *err_dev,
                          const RepDebug *dbg = nullptr) {
    cudaStream_t s = A.stream();
    const int32_t n = L.n;
    // pins(p,e), D(p), saving(v)
    Plist PL;
    PL.p = A.get<int32_t>(L.np);
    PL.cnt = A.get<int32_t>(L.np);
    PL.cin = A.get<int32_t>(L.np);
    PL.lam = A.get<int32_t>(L.e);
    int32_t *D0 = A.get<int32_t>(nparts);
    long long *saving = A.get<long long>(n);
    long long *psize = A.get<long long>(nparts);
    HPC(cudaMemsetAsync(D0, 0, sizeof(int32_t) * nparts, s));
    HPC(cudaMemsetAsync(saving, 0, sizeof(long long) * n, s));
    HPC(cudaMemsetAsync(psize, 0, sizeof(long long) * nparts, s));
    build_plist(L, w, rho, max_e, PL, D0, saving, A);
    k_psize<<<grid_of(n, 256), 256, 0, s>>>(rho, L.size, n, psize);
    HP_LAUNCH_CHECK();

    // moves in isolation (Eq. 13) for nodes that can spare a cut
    int32_t *cnts = A.get<int32_t>(8);
    HPC(cudaMemsetAsync(cnts, 0, 8 * sizeof(int32_t), s));
    int32_t *cl = A.get<int32_t>(n);
    k_candidates<<<grid_of(n, 256), 256, 0, s>>>(saving, n, cl, cnts + 0);
    HP_LAUNCH_CHECK();
    Moves M;
    M.node = A.get<int32_t>(n);
    M.src = A.get<int32_t>(n);
    M.dst = A.get<int32_t>(n);
    M.gain = A.get<long long>(n);
    M.count = cnts + 1;
    int32_t hc[8];
    fetch_bytes(hc, cnts, sizeof hc, s);
    GainArgs G{L.off, L.ioff, L.inc, w, rho, L.size, psize, saving, wns, PL, P.omega, second_half, M};
    if (hc[0] > 0) {
        uint32_t cap = 2048;
        if (P.o.debug_table_cap > 0) cap = (uint32_t)P.o.debug_table_cap;
        size_t sm = (size_t)cap * 12;
        HPC(cudaFuncSetAttribute(k_gains_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        int occ = 0;
        HPC(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gains_smem, GN_T, sm));
        int32_t *ovf = A.get<int32_t>(hc[0]);
        int grid = std::max(1, std::min<int>(hc[0], num_sms() * std::max(occ, 1)));
        k_gains_smem<<<grid, GN_T, sm, s>>>(G, cl, hc[0], cap, ovf, cnts + 2);
        HP_LAUNCH_CHECK();
        int32_t novf = fetch<int32_t>(cnts + 2, s);
        if (novf > 0) {
            uint32_t gcap = pow2_at_least(2 * (int64_t)nparts + 2);
            int nb = std::min<int>(novf, num_sms() * 2);
            int32_t *gk = A.get<int32_t>((int64_t)nb * gcap);
            long long *gc = A.get<long long>((int64_t)nb * gcap);
            k_gains_global<<<nb, GN_T, 0, s>>>(G, ovf, novf, gcap, gk, gc, cl, cnts + 3);
            HP_LAUNCH_CHECK();
            if (fetch<int32_t>(cnts + 3, s)) throw Error(HP_ERR_INTERNAL, "gain table overflow");
            A.release(gk);
            A.release(gc);
        }
        A.release(ovf);
    }
    const int32_t m = fetch<int32_t>(M.count, s);
    if (dbg) *dbg->m = m;
    A.release(cl);
    A.release(saving);
    int32_t applied = 0;
    if (m > 0) {
        // sort (p_s asc, gain desc, node asc)
        unsigned long long *gm = (unsigned long long *)A.get<long long>(1);
        HPC(cudaMemsetAsync(gm, 0, sizeof(long long), s));
        k_max_gain<<<grid_of(m, 256), 256, 0, s>>>(M.gain, m, gm);
        HP_LAUNCH_CHECK();
        const long long gmax = (long long)fetch<unsigned long long>(gm, s);
        const int nb = bits_for((uint64_t)std::max(n - 1, 1)), gb = bits_for((uint64_t)gmax),
                  sb = bits_for((uint64_t)std::max(nparts - 1, 1));
        uint64_t *keys = A.get<uint64_t>(m);
        uint32_t *idx = A.get<uint32_t>(m);
        if (sb + gb + nb <= 64) {
            k_move_keys<<<grid_of(m, 256), 256, 0, s>>>(M, M.count, gmax, gb, nb, keys, idx);
            HP_LAUNCH_CHECK();
            radix_sort(keys, idx, m, sb + gb + nb, A);
        } else {
            iota_i32(reinterpret_cast<int32_t *>(idx), m, s);
            const int fb[3] = {nb, gb, sb};
            for (int f = 0; f < 3; f++) {
                k_field_keys<<<grid_of(m, 256), 256, 0, s>>>(M, m, f, gmax, keys, idx);
                HP_LAUNCH_CHECK();
                radix_sort(keys, idx, m, fb[f], A);
            }
        }
        Moves S;
        S.node = A.get<int32_t>(m);
        S.src = A.get<int32_t>(m);
        S.dst = A.get<int32_t>(m);
        S.gain = A.get<long long>(m);
        S.count = M.count;
        k_gather_moves<<<grid_of(m, 256), 256, 0, s>>>(M, idx, m, S);
        HP_LAUNCH_CHECK();
        A.release(keys);
        A.release(idx);
        if (dbg) {
            HPC(cudaMemcpyAsync(dbg->node, S.node, sizeof(int32_t) * m, cudaMemcpyDeviceToDevice, s));
            HPC(cudaMemcpyAsync(dbg->src, S.src, sizeof(int32_t) * m, cudaMemcpyDeviceToDevice, s));
            HPC(cudaMemcpyAsync(dbg->dst, S.dst, sizeof(int32_t) * m, cudaMemcpyDeviceToDevice, s));
            HPC(cudaMemcpyAsync(dbg->gain, S.gain, sizeof(long long) * m, cudaMemcpyDeviceToDevice, s));
        }
        A.release(gm);

        // chaining (Sec. VI-C)
        int32_t *pc = A.get<int32_t>(nparts + 1);
        int32_t *first = A.get<int32_t>(nparts + 1);
        HPC(cudaMemsetAsync(pc, 0, sizeof(int32_t) * (nparts + 1), s));
        k_part_count<<<grid_of(m, 256), 256, 0, s>>>(S.src, m, pc);
        HP_LAUNCH_CHECK();
        scan_excl(pc, first, nparts + 1, nullptr, A);
        ChainCtx C;
        C.m = m;
        C.window = P.o.chain_window;
        C.node = S.node;
        C.src = S.src;
        C.dst = S.dst;
        C.size = L.size;
        C.nin = L.nin;
        C.gain = S.gain;
        C.first = first;
        C.pred = A.get<int32_t>(m);
        C.succ = A.get<int32_t>(m);
        C.choice = A.get<int32_t>(m);
        C.pen = A.get<unsigned long long>(m);
        C.minpen = A.get<unsigned long long>(m);
        C.accnode = A.get<int32_t>(m);
        C.linked = cnts + 4;
        fill_i32(C.pred, m, -1, s);
        fill_i32(C.succ, m, -1, s);
        for (int32_t r = 0; r < P.o.chain_rounds; r++) {
            HPC(cudaMemsetAsync(C.minpen, 0xff, sizeof(unsigned long long) * m, s));
            fill_i32(C.accnode, m, -1, s);
            HPC(cudaMemsetAsync(C.linked, 0, sizeof(int32_t), s));
            k_choose<<<grid_of(m, 128), 128, 0, s>>>(C);
            HP_LAUNCH_CHECK();
            k_accept_min<<<grid_of(m, 256), 256, 0, s>>>(C);
            HP_LAUNCH_CHECK();
            k_accept_id<<<grid_of(m, 256), 256, 0, s>>>(C);
            HP_LAUNCH_CHECK();
            k_link<<<grid_of(m, 256), 256, 0, s>>>(C);
            HP_LAUNCH_CHECK();
            if (!fetch<int32_t>(C.linked, s)) break;
        }
        A.release(C.choice);
        A.release(C.pen);
        A.release(C.minpen);
        A.release(C.accnode);
        A.release(pc);
        A.release(first);

        // chains in order of (total gain desc, head node asc)
        SeqCtx Q;
        Q.m = m;
        Q.node = S.node;
        Q.pred = C.pred;
        Q.succ = C.succ;
        Q.gain = S.gain;
        Q.chain = A.get<int32_t>(m);
        Q.pos = A.get<int32_t>(m);
        Q.clen = A.get<int32_t>(m);
        Q.cgain = A.get<long long>(m);
        Q.err = err_dev;
        HPC(cudaMemsetAsync(Q.cgain, 0, sizeof(long long) * m, s));
        fill_i32(Q.chain, m, -1, s);
        k_path_heads<<<grid_of(m, 256), 256, 0, s>>>(Q);
        HP_LAUNCH_CHECK();
        k_cycle_heads<<<grid_of(m, 256), 256, 0, s>>>(Q);
        HP_LAUNCH_CHECK();
        int32_t *hflag = A.get<int32_t>(m);
        int32_t *hpos = A.get<int32_t>(m + 1);
        k_head_flags<<<grid_of(m, 256), 256, 0, s>>>(Q.chain, m, hflag);
        HP_LAUNCH_CHECK();
        scan_excl(hflag, hpos, m, hpos + m, A);
        const int32_t nh = fetch<int32_t>(hpos + m, s);
        uint32_t *heads = A.get<uint32_t>(nh);
        k_head_compact<<<grid_of(m, 256), 256, 0, s>>>(hflag, hpos, m, heads);
        HP_LAUNCH_CHECK();
        {
            unsigned long long *cg = (unsigned long long *)A.get<long long>(1);
            HPC(cudaMemsetAsync(cg, 0, sizeof(long long), s));
            k_max_gain<<<grid_of(m, 256), 256, 0, s>>>(Q.cgain, m, cg);  // chain gains are >= 0 at heads, 0 elsewhere
            HP_LAUNCH_CHECK();
            const long long cgmax = (long long)fetch<unsigned long long>(cg, s);
            const int cgb = bits_for((uint64_t)cgmax);
            uint64_t *hk = A.get<uint64_t>(nh);
            if (cgb + nb <= 64) {
                k_head_keys<<<grid_of(nh, 256), 256, 0, s>>>(heads, nh, Q.cgain, S.node, cgmax, nb, -1, hk);
                HP_LAUNCH_CHECK();
                radix_sort(hk, heads, nh, cgb + nb, A);
            } else {
                for (int f = 0; f < 2; f++) {
                    k_head_keys<<<grid_of(nh, 256), 256, 0, s>>>(heads, nh, Q.cgain, S.node, cgmax, nb, f, hk);
                    HP_LAUNCH_CHECK();
                    radix_sort(hk, heads, nh, f == 0 ? nb : cgb, A);
                }
            }
            A.release(hk);
            A.release(cg);
        }
        int32_t *lens = A.get<int32_t>(nh + 1);
        int32_t *starts = A.get<int32_t>(nh + 1);
        k_chain_lens<<<grid_of(nh, 256), 256, 0, s>>>(heads, nh, Q.clen, lens);
        HP_LAUNCH_CHECK();
        scan_excl(lens, starts, nh, nullptr, A);
        int32_t *cstart = A.get<int32_t>(m);
        k_chain_start<<<grid_of(nh, 256), 256, 0, s>>>(heads, nh, starts, cstart);
        HP_LAUNCH_CHECK();
        int32_t *seqpos = A.get<int32_t>(m);
        int32_t *seqmove = A.get<int32_t>(m);
        k_seq_pos<<<grid_of(m, 256), 256, 0, s>>>(Q.chain, Q.pos, cstart, m, seqpos, seqmove);
        HP_LAUNCH_CHECK();
        if (dbg) HPC(cudaMemcpyAsync(dbg->seq, seqmove, sizeof(int32_t) * m, cudaMemcpyDeviceToDevice, s));
        A.release(lens);
        A.release(starts);
        A.release(cstart);
        A.release(heads);
        A.release(hflag);
        A.release(hpos);
        A.release(Q.chain);
        A.release(Q.pos);
        A.release(Q.clen);
        A.release(Q.cgain);
        A.release(C.pred);
        A.release(C.succ);

        // in-sequence gains and distinct-inbound events
        int32_t *evc = A.get<int32_t>(m);
        int32_t *evoff = A.get<int32_t>(m + 1);
        k_ev_count<<<grid_of(m, 256), 256, 0, s>>>(seqmove, S.node, L.ioff, m, evc);
        HP_LAUNCH_CHECK();
        scan_excl(evc, evoff, m, evoff + m, A);
        const int32_t nev = fetch<int32_t>(evoff + m, s);
        const int e_bits = bits_for((uint64_t)std::max(L.e - 1, 1));
        const int p_bits = bits_for((uint64_t)std::max(nparts - 1, 1));
        const int k_bits = bits_for((uint64_t)std::max(m - 1, 1));
        if (e_bits + p_bits + k_bits > 64) throw Error(HP_ERR_INTERNAL, "event key wider than 64 bits");
        unsigned long long *gseq = (unsigned long long *)A.get<long long>(m);
        HPC(cudaMemsetAsync(gseq, 0, sizeof(long long) * m, s));
        uint64_t *dkeys = A.get<uint64_t>(nev);
        int32_t *dvals = A.get<int32_t>(nev);
        if (nev > 0) {
            uint64_t *ek = A.get<uint64_t>(nev);
            uint32_t *ev = A.get<uint32_t>(nev);
            EvCtx E{m, e_bits, p_bits, k_bits, seqmove, S.node, S.src, S.dst, L.ioff, L.inc, L.nin, evoff, ek, ev};
            k_ev_gen<<<grid_of(m, 128), 128, 0, s>>>(E);
            HP_LAUNCH_CHECK();
            radix_sort(ek, ev, nev, e_bits + p_bits + k_bits, A);
            WalkCtx W{nev, p_bits, k_bits, ek, ev, L.off, w, PL, gseq, dkeys, dvals, cnts + 5};
            k_ev_walk<<<grid_of(nev, 256), 256, 0, s>>>(W);
            HP_LAUNCH_CHECK();
            A.release(ek);
            A.release(ev);
        }
        A.release(evc);
        A.release(evoff);
        const int32_t nd = fetch<int32_t>(cnts + 5, s);

        // validity of every prefix (Sec. VI-D)
        const int64_t nv = (int64_t)nd + 2 * (int64_t)m;
        uint64_t *vk = A.get<uint64_t>(nv);
        uint32_t *vi = A.get<uint32_t>(nv);
        long long *vds = A.get<long long>(nv);
        int32_t *vdd = A.get<int32_t>(nv);
        if (nd > 0) {
            k_d_events<<<grid_of(nd, 256), 256, 0, s>>>(dkeys, dvals, nd, vk, vds, vdd);
            HP_LAUNCH_CHECK();
        }
        k_size_events<<<grid_of(m, 256), 256, 0, s>>>(seqmove, S.node, S.src, S.dst, L.size, m, k_bits, vk, vds, vdd,
                                                      nd);
        HP_LAUNCH_CHECK();
        iota_i32(reinterpret_cast<int32_t *>(vi), nv, s);
        radix_sort(vk, vi, nv, p_bits + k_bits, A);
        int32_t *viol = A.get<int32_t>(m);
        HPC(cudaMemsetAsync(viol, 0, sizeof(int32_t) * m, s));
        ValCtx V{nv, k_bits, vk, vi, vds, vdd, psize, D0, P.omega, P.delta, viol};
        k_val_walk<<<grid_of(nv, 256), 256, 0, s>>>(V);
        HP_LAUNCH_CHECK();
        k_initial_bad<<<grid_of(nparts, 256), 256, 0, s>>>(psize, D0, nparts, P.omega, P.delta, cnts + 6);
        HP_LAUNCH_CHECK();
        long long *bgain = A.get<long long>(1);
        k_best_prefix<<<1, 1024, 0, s>>>(gseq, viol, m, cnts + 6, cnts + 7, bgain);
        HP_LAUNCH_CHECK();
        k_apply<<<grid_of(m, 256), 256, 0, s>>>(seqmove, S.node, S.dst, cnts + 7, rho);
        HP_LAUNCH_CHECK();
        applied = fetch<int32_t>(cnts + 7, s);
        if (dbg) {
            HPC(cudaMemcpyAsync(dbg->gseq, gseq, sizeof(long long) * m, cudaMemcpyDeviceToDevice, s));
            HPC(cudaMemcpyAsync(dbg->best_gain, bgain, sizeof(long long), cudaMemcpyDeviceToDevice, s));
        }
        A.release(vk);
        A.release(vi);
        A.release(vds);
        A.release(vdd);
        A.release(viol);
        A.release(bgain);
        A.release(dkeys);
        A.release(dvals);
        A.release(gseq);
        A.release(seqpos);
        A.release(seqmove);
        A.release(S.node);
        A.release(S.src);
        A.release(S.dst);
        A.release(S.gain);
    }
    A.release(M.node);
    A.release(M.src);
    A.release(M.dst);
    A.release(M.gain);
    A.release(cnts);
    A.release(PL.p);
    A.release(PL.cnt);
    A.release(PL.cin);
    A.release(PL.lam);
    A.release(D0);
    A.release(psize);
    return applied;
}

int32_t refine_rep_debug(const Level &L, const int32_t *w, int32_t nparts, const Params &P, int32_t *rho,
                         int second_half, Arena &A, uint32_t *err_dev, const RepDebug &dbg) {
    cudaStream_t s = A.stream();
    int32_t *maxe = A.get<int32_t>(1);
    HPC(cudaMemsetAsync(maxe, 0, sizeof(int32_t), s));
    if (L.e > 0) {
        k_max_edge<<<grid_of(L.e, 256), 256, 0, s>>>(L.off, L.e, maxe);
        HP_LAUNCH_CHECK();
    }
    const int32_t max_e = fetch<int32_t>(maxe, s);
    long long *wns = A.get<long long>(std::max(L.n, 1));
    if (L.n > 0) {
        k_wns<<<grid_of(L.n, 256), 256, 0, s>>>(L.off, L.ioff, L.inc, w, L.n, wns);
        HP_LAUNCH_CHECK();
    }
    *dbg.m = 0;
    int32_t k = L.n > 0 ? refine_rep(L, w, nparts, P, rho, second_half, max_e, wns, A, err_dev, &dbg) : 0;
    A.release(wns);
    A.release(maxe);
    return k;
}

RefineOut refine_level(const Level &L, const int32_t *w, int32_t nparts, const Params &P, int32_t *rho, Arena &A,
                       uint32_t *err_dev) {
    cudaStream_t s = A.stream();
    RefineOut out;
    if (L.n == 0 || P.o.theta == 0) return out;
    int32_t *maxe = A.get<int32_t>(1);
    HPC(cudaMemsetAsync(maxe, 0, sizeof(int32_t), s));
    if (L.e > 0) {
        k_max_edge<<<grid_of(L.e, 256), 256, 0, s>>>(L.off, L.e, maxe);
        HP_LAUNCH_CHECK();
    }
    const int32_t max_e = fetch<int32_t>(maxe, s);
    A.release(maxe);
    long long *wns = A.get<long long>(L.n);
    k_wns<<<grid_of(L.n, 256), 256, 0, s>>>(L.off, L.ioff, L.inc, w, L.n, wns);
    HP_LAUNCH_CHECK();
    const int32_t half = P.o.theta / 2;
    for (int32_t rep = 0; rep < P.o.theta; rep++) {
        int32_t k = refine_rep(L, w, nparts, P, rho, rep >= half, max_e, wns, A, err_dev);
        out.reps++;
        out.moves += k;
        if (k == 0) {
            if (rep < half) rep = half - 1;
            else break;
        }
    }
    A.release(wns);
    return out;
}

}  // namespace hp

namespace hp {

// ---------------------------------------------------------------- final statistics
__global__ void k_part_sizes(const int32_t *part, int32_t n, long long *psize) {
    GRID_STRIDE(v, (int64_t)n) atomicAdd((unsigned long long *)&psize[part[v]], 1ull);
}
__global__ void k_part_max(const long long *psize, const int32_t *D, int32_t nparts, int32_t omega, int32_t delta,
                           long long *out) {
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
        k_max_edge<<<grid_of(L.e, 256), 256, 0, s>>>(L.off, L.e, maxe);
        HP_LAUNCH_CHECK();
        int32_t me = fetch<int32_t>(maxe, s);
        Plist PL;
        PL.p = A.get<int32_t>(L.np);
        PL.cnt = A.get<int32_t>(L.np);
        PL.cin = A.get<int32_t>(L.np);
        PL.lam = A.get<int32_t>(L.e);
        build_plist(L, w, part, me, PL, D, nullptr, A);
        k_objective<<<grid_of(L.e, 256), 256, 0, s>>>(PL.lam, w, L.e, (unsigned long long *)out,
                                                      (unsigned long long *)(out + 1));
        HP_LAUNCH_CHECK();
        A.release(PL.p);
        A.release(PL.cnt);
        A.release(PL.cin);
        A.release(PL.lam);
        A.release(maxe);
    }
    k_part_sizes<<<grid_of(L.n, 256), 256, 0, s>>>(part, L.n, psize);
    HP_LAUNCH_CHECK();
    k_part_max<<<grid_of(nparts, 256), 256, 0, s>>>(psize, D, nparts, omega, delta, (long long *)out);
    HP_LAUNCH_CHECK();
    A.release(D);
    A.release(psize);
}

}  // namespace hp
