// hp_coarsen.cu -- one coarsening level: candidate-pair proposal (Sec. V-C,
// Eq. 5-6, deterministic noise, best-effort pairing of nodes without a valid
// neighbour) and maximum-weight matching on the proposal pseudo-forest
// (Sec. V-D, Eq. 7-12), repeated for Pi proposal graphs.
//
// The proposal fuses neighbour deduplication with the eta/inter histogram:
// one CTA per node walks I(n) and the pins of every incident hyperedge and
// accumulates into a shared-memory table (direct-indexed when the level has
// at most 16384 nodes, open-addressing otherwise; nodes whose neighbourhood
// outgrows the table are redone with a larger table and finally with a table
// in global memory).  Sums and counts are integers, so the result does not
// depend on the order of the atomic updates.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>

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

constexpr int PT = 256;          // proposal CTA size
constexpr int DENSE_N = 16384;   // direct-indexed table up to this many nodes (12 B per node)

// ---------------------------------------------------------------- noise
// SplitMix64 finaliser (Steele, Lea, Flood 2014) keyed by (seed, level,
// min(n,m), max(n,m)), reduced modulo cap+1: symmetric by construction.
__device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t pair_noise(uint64_t level_key, int32_t a, int32_t b, uint64_t cap) {
    uint32_t lo = (uint32_t)min(a, b), hi = (uint32_t)max(a, b);
    uint64_t h = sm64_mix(level_key ^ (((uint64_t)lo << 32) | (uint64_t)hi));
    return h % (cap + 1);
}

struct PropCtx {
    int32_t n, pi;
    const int32_t *off, *pin, *nsrc, *size, *ioff, *inc, *nin;
    const uint64_t *q;
    const uint64_t *cap;   // device scalar
    uint64_t level_key;
    int32_t omega, delta;
    int32_t *cand;         // [n*pi]
    uint64_t *cscore;      // [n*pi]
    int32_t *nbcnt;        // [n] unique neighbours found (those that pass the size filter)
    const int32_t *canon;  // [e] hyperedges with equal destination lists share a value (or null)
    const int32_t *canon_on;   // device scalar: nonzero when canon groups hyperedges (used only with canon)
    int32_t size_filter;   // 1: neighbours m with size(v) + size(m) > Omega are not entered in v's table
};

// The destination-list groups when they pay: a level whose lists are all
// distinct (no group of two) walks every hyperedge alone, without the
// CTA-wide queue of group walks.  Result-neutral: the table sums are the same.
__device__ __forceinline__ const int32_t *dst_groups_of(const PropCtx &C) {
    return (C.canon && *C.canon_on) ? C.canon : nullptr;
}

// A neighbour that fails the size half of Eq. 6 can never be a candidate,
// so with the filter on it is not entered in the table at all.  The count of
// entered neighbours then bounds the size-valid neighbours of the cluster at
// the next level (sizes only grow), and a node whose bound is 0 has no valid
// neighbour: result-neutral either way.
__device__ __forceinline__ int32_t size_slack(const PropCtx &C, int32_t v) {
    return C.size_filter ? C.omega - C.size[v] : INT32_MAX;
}
__device__ __forceinline__ bool size_ok(const PropCtx &C, int32_t slack, int32_t m) {
    return !C.size_filter || C.size[m] <= slack;
}

// ---------------------------------------------------------------- per-level weights
__global__ void k_level_q(const int32_t *off, const int32_t *w, int32_t e, uint64_t *q, unsigned long long *sum) {
    HP_KERNEL_ENTER();
    __shared__ unsigned long long s;
    if (threadIdx.x == 0) s = 0;
    __syncthreads();
    unsigned long long loc = 0;
    GRID_STRIDE(i, (int64_t)e) {
        // floor(w 2^24 / |e|): the numerator is below 2^41 and the divisor
        // below 2^31, so the correctly rounded double quotient of a
        // non-integer ratio is never rounded across an integer
        const double num = (double)((uint64_t)w[i] << 24), den = (double)(off[i + 1] - off[i]);
        const uint64_t qi = (uint64_t)floor(num / den);
        q[i] = qi;
        loc += qi;
    }
    for (int o = 16; o > 0; o >>= 1) loc += __shfl_down_sync(0xffffffffu, loc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&s, loc);
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(sum, s);
}

// the level's counters, node sums and tier counts start at zero (one launch
// instead of four memsets, which would each end the overlap of a launch with
// its predecessor)
__global__ void k_level_start(LevelBox *box, long long *nsum, long long *vis, int32_t n, int32_t *cnt) {
    HP_KERNEL_ENTER();
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t0 < (int64_t)(sizeof(LevelBox) / sizeof(uint32_t))) reinterpret_cast<uint32_t *>(box)[t0] = 0u;
    if (t0 < 8) cnt[t0] = 0;
    GRID_STRIDE(v, (int64_t)n) {
        nsum[v] = 0;
        vis[v] = 0;
    }
}

// per incidence entry (e, v): sums over I(v) of |e| - 1 (bound on |N(v)|)
// and |e| (pins the traversal of v visits), reduced per run of equal v
// inside a warp, so hub nodes with huge incidence lists spread over threads
__global__ void k_node_sums(const int32_t *off, const int32_t *inc, const int32_t *inode, int64_t np,
                            long long *nsum, long long *vis, unsigned long long *visits) {
    HP_KERNEL_ENTER();
    const int lane = threadIdx.x & 31;
    const int64_t wbase = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) << 5;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long loc = 0;
    for (int64_t base = wbase; base < np; base += stride) {
        const int64_t t = base + lane;
        const bool valid = t < np;
        const int32_t v = valid ? inode[t] : -1 - lane;
        long long sz = 0;
        if (valid) {
            const int32_t e = inc[t];
            sz = off[e + 1] - off[e];
            loc += (unsigned long long)sz;
        }
        long long a = valid ? sz - 1 : 0, b = sz;
        bool tail = warp_run_sum(v, a);
        warp_run_sum(v, b);
        if (valid && tail) {
            atomicAdd((unsigned long long *)&nsum[v], (unsigned long long)a);
            atomicAdd((unsigned long long *)&vis[v], (unsigned long long)b);
        }
    }
    for (int o = 16; o > 0; o >>= 1) loc += __shfl_down_sync(0xffffffffu, loc, o);
    if (lane == 0) atomicAdd(visits, loc);
}

__global__ void k_node_bounds(const long long *nsum, int32_t n, int32_t *bound, LevelBox *box, int32_t e,
                              int32_t permille) {
    HP_KERNEL_ENTER();
    // the noise cap of the level from the sum of q (complete: k_level_q ran before)
    if (blockIdx.x == 0 && threadIdx.x == 0)
        box->cap = e > 0 ? (uint64_t)((box->qsum / (unsigned long long)e) * (unsigned long long)permille / 1000ull)
                         : 0ull;
    GRID_STRIDE(v, (int64_t)n) {
        long long b = bound[v];
        if (nsum[v] < b) b = nsum[v];
        if (n - 1 < b) b = n - 1;
        bound[v] = (int32_t)b;
    }
}

// ---------------------------------------------------------------- top-Pi selection
struct Cand {
    uint64_t eta;
    int32_t id;
};
__device__ __forceinline__ bool cand_gt(const Cand &a, const Cand &b) {
    return a.eta > b.eta || (a.eta == b.eta && a.id > b.id);
}

// x added to the 64-bit counter at p with two 32-bit atomics: the low word's
// carry goes to the high word, so the counter ends equal to the exact sum
// (all updates of p use this form).
__device__ __forceinline__ void add_u64_split(unsigned long long *p, unsigned long long x) {
    uint32_t *w = reinterpret_cast<uint32_t *>(p);
    const uint32_t xl = (uint32_t)x, xh = (uint32_t)(x >> 32);
    const uint32_t old = atomicAdd(&w[0], xl);
    const uint32_t hi = xh + (uint32_t)((uint32_t)(old + xl) < old);
    if (hi) atomicAdd(&w[1], hi);
}

template <int PIMAX> struct TopList {
    Cand c[PIMAX];
    __device__ void init() {
#pragma unroll
        for (int i = 0; i < PIMAX; i++) c[i] = Cand{0, -1};
    }
    __device__ void push(Cand x) {
#pragma unroll
        for (int i = 0; i < PIMAX; i++) {
            if (cand_gt(x, c[i])) {
                Cand t = c[i];
                c[i] = x;
                x = t;
            }
        }
    }
    __device__ void pop() {
#pragma unroll
        for (int i = 0; i < PIMAX - 1; i++) c[i] = c[i + 1];
        c[PIMAX - 1] = Cand{0, -1};
    }
};

// block-wide: write the pi best of the per-thread lists to cand/cscore of v.
// Each warp first extracts its own pi best by shuffles (no barrier); warp 0
// then merges the warps' lists from s_top (32 * PIMAX entries).
template <int PIMAX>
__device__ __forceinline__ Cand warp_pop_best(TopList<PIMAX> &tl) {
    Cand best = tl.c[0];
    int owner = threadIdx.x & 31;
    for (int o = 16; o > 0; o >>= 1) {
        Cand ob{__shfl_xor_sync(0xffffffffu, best.eta, o), __shfl_xor_sync(0xffffffffu, best.id, o)};
        const int oo = __shfl_xor_sync(0xffffffffu, owner, o);
        if (cand_gt(ob, best) || (ob.id == best.id && oo < owner)) {
            best = ob;
            owner = oo;
        }
    }
    if (best.id >= 0 && (int)(threadIdx.x & 31) == owner) tl.pop();
    return best;
}
template <int PIMAX>
__device__ void block_emit_top(TopList<PIMAX> &tl, const PropCtx &C, int32_t v, Cand *s_top) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int r = 0; r < C.pi; r++) {
        const Cand b = warp_pop_best(tl);
        if (lane == 0) s_top[wid * PIMAX + r] = b;
    }
    __syncthreads();
    if (wid == 0) {
        TopList<PIMAX> m;
        m.init();
        for (int i = lane; i < nw * C.pi; i += 32) m.push(s_top[(i / C.pi) * PIMAX + (i % C.pi)]);
        for (int r = 0; r < C.pi; r++) {
            const Cand b = warp_pop_best(m);
            if (lane == 0) {
                C.cand[(int64_t)v * C.pi + r] = b.id;
                C.cscore[(int64_t)v * C.pi + r] = b.id >= 0 ? b.eta : 0;
            }
        }
    }
    __syncthreads();
}

// Lists longer than four (PIMAX > 4) are emitted in rounds of four so that
// every thread keeps a TopList<4> only: round r writes entries r0..r0+nr-1
// of v's list, the nr best candidates strictly below `thr` (the last entry
// of the previous round).  Returns the last entry written, the same in every
// thread of the block; {0, -1} once the candidates run out, below which
// nothing lies.
constexpr int EMIT_W = 4;
__device__ Cand block_emit_range(TopList<EMIT_W> &tl, const PropCtx &C, int32_t v, Cand *s_top, int r0, int nr,
                                 Cand *s_last) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int r = 0; r < nr; r++) {
        const Cand b = warp_pop_best(tl);
        if (lane == 0) s_top[wid * EMIT_W + r] = b;
    }
    __syncthreads();
    if (wid == 0) {
        TopList<EMIT_W> m;
        m.init();
        for (int i = lane; i < nw * nr; i += 32) m.push(s_top[(i / nr) * EMIT_W + (i % nr)]);
        Cand b{0, -1};
        for (int r = 0; r < nr; r++) {
            b = warp_pop_best(m);
            if (lane == 0) {
                C.cand[(int64_t)v * C.pi + r0 + r] = b.id;
                C.cscore[(int64_t)v * C.pi + r0 + r] = b.id >= 0 ? b.eta : 0;
            }
        }
        if (lane == 0) *s_last = b;
    }
    __syncthreads();
    return *s_last;
}

__device__ __forceinline__ bool pair_valid(const PropCtx &C, int32_t v, int32_t m, int32_t inter) {
    if ((int64_t)C.size[v] + C.size[m] > C.omega) return false;
    return (int64_t)C.nin[v] + C.nin[m] - inter <= C.delta;
}

__device__ __forceinline__ int32_t block_sum_i32(int32_t x, int32_t *s_tmp) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) s_tmp[threadIdx.x >> 5] = x;
    __syncthreads();
    int32_t t = 0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += s_tmp[k];
    __syncthreads();
    return t;
}

// One chunk of v's incidence for the calling warp: lane l takes the
// hyperedge at incidence index t = base + l (none when t >= deg).
// Hyperedges of 2..32 pins: the j-th pins of the warp's hyperedges are
// combined by neighbour (match_any) and one table update per distinct
// neighbour carries the warp's sums of q(e) and of the inbound-overlap
// counts; q(e) <= 2^40 is summed as two 21-bit halves so that 32-bit warp
// reductions cannot overflow.  Larger hyperedges: each lane inserts its own
// source pins; the destination pins are walked once per group of the warp's
// hyperedges with equal destination lists (C.canon; every hyperedge alone
// when it is null), carrying the group's sum of q(e) and, when v is one of
// those destinations, the group's size as the inbound overlap.  That walk is
// handed to big(e, qsum, icnt) when it is given, else the warp takes the
// groups one at a time, lanes over pins.
template <class Ins, class Big>
__device__ __forceinline__ void warp_chunk(const PropCtx &C, int32_t v, int32_t i0, int32_t deg, int32_t nin_v,
                                           int32_t t, Ins &ins, Big *big) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    int32_t e = -1, a = 0, sz = 0, dst0 = 0;
    unsigned long long qe = 0;
    bool vin = false;
    if (t < deg) {
        e = C.inc[i0 + t];
        a = C.off[e];
        sz = C.off[e + 1] - a;
        if (sz < 2) {
            sz = 0;
        } else {
            dst0 = a + C.nsrc[e];
            qe = C.q[e];
            vin = t < nin_v;
        }
    }
    const bool large = sz > 32;
    const int32_t len = large ? 0 : sz;
    const int32_t slack = size_slack(C, v);
    const int jmax = (int)__reduce_max_sync(FULL, (unsigned)len);
    for (int j = 0; j < jmax; j++) {
        int32_t m = j < len ? C.pin[a + j] : -1;
        if (m == v) m = -1;
        const unsigned g = __match_any_sync(FULL, m);
        const bool on = m >= 0;
        const unsigned lo = __reduce_add_sync(g, on ? (unsigned)(qe & 0x1FFFFFull) : 0u);
        const unsigned hi = __reduce_add_sync(g, on ? (unsigned)(qe >> 21) : 0u);
        const unsigned ic = __reduce_add_sync(g, (on && vin && a + j >= dst0) ? 1u : 0u);
        if (on && (g & lt) == 0u && size_ok(C, slack, m))
            ins(m, (unsigned long long)lo + ((unsigned long long)hi << 21), ic);
    }
    const unsigned bigm = __ballot_sync(FULL, large);
    if (!bigm) return;
    // groups of large hyperedges with equal destination lists
    const int32_t *canon = dst_groups_of(C);
    const int32_t key = large ? (canon ? canon[e] : e) : -1 - lane;
    const unsigned grp = __match_any_sync(FULL, key);
    const unsigned qlo = __reduce_add_sync(grp, large ? (unsigned)(qe & 0x1FFFFFull) : 0u);
    const unsigned qhi = __reduce_add_sync(grp, large ? (unsigned)(qe >> 21) : 0u);
    const unsigned long long qsum = (unsigned long long)qlo + ((unsigned long long)qhi << 21);
    const uint32_t icnt = vin ? (uint32_t)__popc(grp) : 0u;
    const bool lead = large && (grp & lt) == 0u;
    if (large)
        for (int32_t j = a; j < dst0; j++) {
            const int32_t m = C.pin[j];
            if (m != v && size_ok(C, slack, m)) ins(m, qe, 0u);
        }
    if (big) {
        if (lead) (*big)(e, qsum, icnt);
        return;
    }
    unsigned lm = __ballot_sync(FULL, lead);
    while (lm) {
        const int l = __ffs(lm) - 1;
        lm &= lm - 1;
        const int32_t ld0 = __shfl_sync(FULL, dst0, l), lb = __shfl_sync(FULL, a, l) + __shfl_sync(FULL, sz, l);
        const unsigned long long lq = __shfl_sync(FULL, qsum, l);
        const uint32_t lc = __shfl_sync(FULL, icnt, l);
        for (int32_t j = ld0 + lane; j < lb; j += 32) {
            const int32_t m = C.pin[j];
            if (m != v && size_ok(C, slack, m)) ins(m, lq, lc);
        }
    }
}

struct NoBig {
    __device__ void operator()(int32_t, unsigned long long, uint32_t) const {}
};

// A warp's walk over all of v's hyperedges.
template <class Ins>
__device__ __forceinline__ void warp_walk(const PropCtx &C, int32_t v, int32_t i0, int32_t deg, int32_t nin_v,
                                          Ins ins) {
    for (int32_t base = 0; base < deg; base += 32)
        warp_chunk(C, v, i0, deg, nin_v, base + (int32_t)(threadIdx.x & 31), ins, (NoBig *)nullptr);
}

// Shared-memory queue of destination walks of one CTA: blockDim.x entries.
struct BigQueue {
    int32_t *e;
    unsigned long long *q;
    uint32_t *c;
    int32_t *n;   // == 0 on entry and on exit of cta_walk
};

// A CTA's walk over all of v's hyperedges in chunks of blockDim.x: small
// ones and source pins as above, destination walks of large ones queued in
// shared memory and then taken a warp each, lanes over pins, so that every
// warp gets a share of them.  Stops early (for every thread) once *stop is
// set.
//
// On levels without destination-list groups (small hyperedges, the coarse
// levels, nets whose lists are all distinct) every warp walks its own
// contiguous share of ceil(deg / warps) incidence entries, 32 at a time, with
// no CTA barrier until the end, and walks its large hyperedges itself: even
// a node of a few dozen hyperedges spreads them over all warps.
template <class Ins>
__device__ void cta_walk(const PropCtx &C, int32_t v, int32_t i0, int32_t deg, int32_t nin_v, const int *stop,
                         BigQueue Q, Ins ins) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (!dst_groups_of(C)) {
        const int32_t share = (deg + nw - 1) / nw, lo = wid * share, hi = min(deg, lo + share);
        for (int32_t base = lo; base < hi; base += 32) {
            if (__any_sync(0xffffffffu, stop ? *(volatile const int *)stop : 0)) break;
            warp_chunk(C, v, i0, deg, nin_v, base + lane < hi ? base + lane : deg, ins, (NoBig *)nullptr);
        }
        __syncthreads();
        return;
    }
    const int32_t slack = size_slack(C, v);
    auto push = [&](int32_t e, unsigned long long qsum, uint32_t icnt) {
        const int32_t i = atomicAdd(Q.n, 1);
        Q.e[i] = e;
        Q.q[i] = qsum;
        Q.c[i] = icnt;
    };
    for (int32_t base = 0; base < deg; base += blockDim.x) {
        if (__syncthreads_or(stop ? *(volatile const int *)stop : 0)) break;
        warp_chunk(C, v, i0, deg, nin_v, base + (int32_t)threadIdx.x, ins, &push);
        __syncthreads();
        const int32_t nb = *(volatile int32_t *)Q.n;
        for (int32_t i = wid; i < nb; i += nw) {
            const int32_t e = Q.e[i];
            const unsigned long long qsum = Q.q[i];
            const uint32_t icnt = Q.c[i];
            const int32_t b = C.off[e + 1];
            // the next pin is loaded before the current one is inserted
            int32_t j = C.off[e] + C.nsrc[e] + lane;
            int32_t mn = j < b ? __ldg(&C.pin[j]) : -1;
            while (j < b) {
                const int32_t m = mn, jn = j + 32;
                mn = jn < b ? __ldg(&C.pin[jn]) : -1;
                if (m != v && size_ok(C, slack, m)) ins(m, qsum, icnt);
                j = jn;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) *Q.n = 0;
    }
    __syncthreads();
}

// ---------------------------------------------------------------- destination-list groups
// canon[e] = one representative of the hyperedges whose destination pin
// lists equal e's (levels of large hyperedges; the proposal walks such lists once per warp
// group).  Lists are hashed, sorted by hash, and equal neighbours in that
// order are confirmed pin by pin, so a hash collision only splits a group.
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}
__global__ void k_dst_hash(const int32_t *off, const int32_t *pin, const int32_t *nsrc, int32_t e, uint32_t *key,
                           uint32_t *val) {
    HP_KERNEL_ENTER();
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5, nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w0; i < e; i += nw) {
        const int32_t d0 = off[i] + nsrc[i], b = off[i + 1];
        uint32_t h = 0;
        for (int32_t j = d0 + lane; j < b; j += 32) h += fmix32((uint32_t)pin[j] ^ ((uint32_t)(j - d0) * 0x9E3779B9u));
        for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
        if (lane == 0) {
            key[i] = fmix32(h ^ (uint32_t)(b - d0));
            val[i] = (uint32_t)i;
        }
    }
}
__global__ void k_dst_runs(const uint32_t *key, const uint32_t *val, const int32_t *off, const int32_t *pin,
                           const int32_t *nsrc, int32_t e, int32_t *newrun) {
    HP_KERNEL_ENTER();
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5, nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w0; i < e; i += nw) {
        bool same = i > 0 && key[i] == key[i - 1];
        if (same) {
            const int32_t x = (int32_t)val[i], y = (int32_t)val[i - 1];
            const int32_t xa = off[x] + nsrc[x], xb = off[x + 1], ya = off[y] + nsrc[y], yb = off[y + 1];
            same = xb - xa == yb - ya;
            for (int32_t k = lane; same && k < xb - xa; k += 32)
                same = __all_sync(__activemask(), pin[xa + k] == pin[ya + k]);
        }
        if (lane == 0) newrun[i] = same ? 0 : 1;
    }
}
__global__ void k_dst_rep(const uint32_t *val, const int32_t *newrun, const int32_t *runpos, int32_t e, int32_t *rep) {
    HP_KERNEL_ENTER();
    GRID_STRIDE(i, (int64_t)e) {
        if (newrun[i]) rep[runpos[i]] = (int32_t)val[i];
    }
}
__global__ void k_dst_canon(const uint32_t *val, const int32_t *newrun, const int32_t *runpos, const int32_t *rep,
                            int32_t e, int32_t *canon) {
    HP_KERNEL_ENTER();
    GRID_STRIDE(i, (int64_t)e) canon[val[i]] = rep[runpos[i] + newrun[i] - 1];
}

// ---------------------------------------------------------------- dense table
// eta[m], inter[m] for every node of the level in shared memory (levels of at
// most DENSE_N nodes, nodes with large neighbourhoods).
template <int PIMAX, int BT>
__global__ void __launch_bounds__(BT) k_propose_dense(PropCtx C, const int32_t *list, const int32_t *count_p) {
    HP_KERNEL_ENTER();
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long *eta = reinterpret_cast<unsigned long long *>(smem);
    uint32_t *inter = reinterpret_cast<uint32_t *>(eta + C.n);
    __shared__ Cand s_top[32 * PIMAX];
    __shared__ int32_t s_qe[BT];
    __shared__ unsigned long long s_qq[BT];
    __shared__ uint32_t s_qc[BT];
    __shared__ int32_t s_nbig;
    __shared__ int32_t s_tmp[32];
    const int32_t count = *count_p;
    if (count == 0) return;
    for (int32_t i = threadIdx.x; i < C.n; i += BT) {
        eta[i] = 0;
        inter[i] = 0;
    }
    if (threadIdx.x == 0) s_nbig = 0;
    __syncthreads();
    const uint64_t cap = *C.cap;
    for (int32_t k = blockIdx.x; k < count; k += gridDim.x) {
        const int32_t v = list[k];
        const int32_t i0 = C.ioff[v], deg = C.ioff[v + 1] - i0, nin_v = C.nin[v];
        cta_walk(C, v, i0, deg, nin_v, nullptr, BigQueue{s_qe, s_qq, s_qc, &s_nbig},
                 [&](int32_t m, unsigned long long eq, uint32_t ic) {
            add_u64_split(&eta[m], eq);
            if (ic) atomicAdd(&inter[m], ic);
        });
        __syncthreads();
        if constexpr (PIMAX <= EMIT_W) {
            TopList<PIMAX> tl;
            tl.init();
            int32_t cnt = 0;
            for (int32_t m = threadIdx.x; m < C.n; m += BT) {
                unsigned long long em = eta[m];
                if (em) {
                    cnt++;
                    int32_t it = (int32_t)inter[m];
                    if (pair_valid(C, v, m, it)) tl.push(Cand{em + pair_noise(C.level_key, v, m, cap), m});
                    eta[m] = 0;
                    inter[m] = 0;
                }
            }
            int32_t tot = block_sum_i32(cnt, s_tmp);
            if (threadIdx.x == 0) C.nbcnt[v] = tot;
            block_emit_top<PIMAX>(tl, C, v, s_top);
        } else {
            Cand thr{~0ull, INT32_MAX};
            for (int r0 = 0; r0 < C.pi; r0 += EMIT_W) {
                TopList<EMIT_W> tl;
                tl.init();
                for (int32_t m = threadIdx.x; m < C.n; m += BT) {
                    const unsigned long long em = eta[m];
                    if (em && pair_valid(C, v, m, (int32_t)inter[m])) {
                        const Cand c{em + pair_noise(C.level_key, v, m, cap), m};
                        if (cand_gt(thr, c)) tl.push(c);
                    }
                }
                thr = block_emit_range(tl, C, v, s_top, r0, min(EMIT_W, C.pi - r0), &s_top[32 * PIMAX - 1]);
            }
            int32_t cnt = 0;
            for (int32_t m = threadIdx.x; m < C.n; m += BT) {
                if (eta[m]) {
                    cnt++;
                    eta[m] = 0;
                    inter[m] = 0;
                }
            }
            int32_t tot = block_sum_i32(cnt, s_tmp);
            if (threadIdx.x == 0) C.nbcnt[v] = tot;
        }
    }
}

// ---------------------------------------------------------------- warp per node
// Nodes whose neighbourhood bound is at most half the per-warp table: one
// warp per node, no block barriers.  Incident hyperedges of up to 32 pins are
// spread over the lanes (one hyperedge per lane), larger ones lane per pin.
constexpr int WP_T = 256;
__device__ __forceinline__ uint32_t hslot_w(int32_t m, uint32_t mask) {
    return mask ? ((uint32_t)m * 0x9E3779B1u) >> __clz(mask) : 0u;   // top bits (Fibonacci hashing)
}
__device__ __forceinline__ void warp_insert(int32_t *keys, unsigned long long *eta, uint32_t *inter, uint32_t mask,
                                            uint32_t cap, int32_t m, unsigned long long qe, uint32_t ninter) {
    uint32_t h = hslot_w(m, mask);
    for (uint32_t probe = 0; probe < cap; probe++) {
        int32_t k = ((volatile int32_t *)keys)[h];
        if (k == -1) {
            int32_t old = atomicCAS(&keys[h], -1, m);
            k = old == -1 ? m : old;
        }
        if (k == m) {
            add_u64_split(&eta[h], qe);
            if (ninter) atomicAdd(&inter[h], ninter);
            return;
        }
        h = (h + 1) & mask;
    }
}
template <int PIMAX>
__global__ void __launch_bounds__(WP_T) k_propose_warp(PropCtx C, const int32_t *list, const int32_t *count_p,
                                                       uint32_t cap) {
    HP_KERNEL_ENTER();
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwb = WP_T / 32;
    unsigned long long *eta = reinterpret_cast<unsigned long long *>(smem) + (size_t)wid * cap;
    uint32_t *inter = reinterpret_cast<uint32_t *>(reinterpret_cast<unsigned long long *>(smem) + (size_t)nwb * cap) +
                      (size_t)wid * cap;
    int32_t *keys = reinterpret_cast<int32_t *>(reinterpret_cast<uint32_t *>(reinterpret_cast<unsigned long long *>(
                                                    smem) + (size_t)nwb * cap) + (size_t)nwb * cap) +
                    (size_t)wid * cap;
    const int32_t count = *count_p;
    if (count == 0) return;
    const uint32_t mask = cap - 1;
    for (uint32_t i = lane; i < cap; i += 32) {
        keys[i] = -1;
        eta[i] = 0;
        inter[i] = 0;
    }
    __syncwarp();
    const uint64_t capn = *C.cap;
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = gw; k < count; k += nw) {
        const int32_t v = list[k];
        const int32_t i0 = C.ioff[v], deg = C.ioff[v + 1] - i0, nin_v = C.nin[v];
        // all incident hyperedges, one per lane, combined across the warp
        warp_walk(C, v, i0, deg, nin_v, [&](int32_t m, unsigned long long eq, uint32_t ic) {
            warp_insert(keys, eta, inter, mask, cap, m, eq, ic);
        });
        __syncwarp();
        // the warp's best entries r0.. of v's list from the lanes' lists
        auto emit = [&](auto &tl, int r0, int nr) {
            Cand last{0, -1};
            for (int r = 0; r < nr; r++) {
                Cand best = tl.c[0];
                int owner = lane;
                for (int o = 16; o > 0; o >>= 1) {
                    Cand ob{__shfl_xor_sync(0xffffffffu, best.eta, o), __shfl_xor_sync(0xffffffffu, best.id, o)};
                    int oo = __shfl_xor_sync(0xffffffffu, owner, o);
                    if (cand_gt(ob, best)) {
                        best = ob;
                        owner = oo;
                    }
                }
                if (lane == 0) {
                    C.cand[(int64_t)v * C.pi + r0 + r] = best.id;
                    C.cscore[(int64_t)v * C.pi + r0 + r] = best.id >= 0 ? best.eta : 0;
                }
                if (best.id >= 0 && lane == owner) tl.pop();
                last = best;
            }
            return last;
        };
        int32_t cnt = 0;
        if constexpr (PIMAX <= EMIT_W) {
            TopList<PIMAX> tl;
            tl.init();
            for (uint32_t h = lane; h < cap; h += 32) {
                const int32_t m = keys[h];
                if (m >= 0) {
                    cnt++;
                    if (pair_valid(C, v, m, (int32_t)inter[h])) tl.push(Cand{eta[h] + pair_noise(C.level_key, v, m, capn), m});
                    keys[h] = -1;
                    eta[h] = 0;
                    inter[h] = 0;
                }
            }
            __syncwarp();
            for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
            if (lane == 0) C.nbcnt[v] = cnt;
            emit(tl, 0, C.pi);
        } else {
            // rounds of four, each below the last entry of the round before
            // the first round stores each neighbour's noised score in its eta
            // slot and its validity in its inter slot, the later rounds only
            // compare
            Cand thr{~0ull, INT32_MAX};
            for (int r0 = 0; r0 < C.pi; r0 += EMIT_W) {
                TopList<EMIT_W> tl;
                tl.init();
                for (uint32_t h = lane; h < cap; h += 32) {
                    const int32_t m = keys[h];
                    if (m < 0) continue;
                    unsigned long long sc = eta[h];
                    bool ok = inter[h] != 0;
                    if (r0 == 0) {
                        ok = pair_valid(C, v, m, (int32_t)inter[h]);
                        if (ok) sc += pair_noise(C.level_key, v, m, capn);
                        eta[h] = sc;
                        inter[h] = ok ? 1u : 0u;
                    }
                    if (ok) {
                        const Cand c{sc, m};
                        if (cand_gt(thr, c)) tl.push(c);
                    }
                }
                thr = emit(tl, r0, min(EMIT_W, C.pi - r0));
            }
            for (uint32_t h = lane; h < cap; h += 32) {
                if (keys[h] >= 0) {
                    cnt++;
                    keys[h] = -1;
                    eta[h] = 0;
                    inter[h] = 0;
                }
            }
            __syncwarp();
            for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
            if (lane == 0) C.nbcnt[v] = cnt;
        }
    }
}

// ---------------------------------------------------------------- hashed table
__device__ __forceinline__ uint32_t hslot(int32_t m, uint32_t mask) {
    return mask ? ((uint32_t)m * 0x9E3779B1u) >> __clz(mask) : 0u;   // top bits (Fibonacci hashing)
}

// Table of `cap` slots at keys/eta/inter (shared or global).  Nodes from
// list[0..count) are processed; a node whose distinct neighbours exceed
// limit is appended to ovf (and its table cleared).
template <int PIMAX>
__device__ void propose_hashed_node(const PropCtx &C, int32_t v, int32_t *keys, unsigned long long *eta,
                                    uint32_t *inter, uint32_t cap, uint32_t limit, int32_t *slots, int32_t *ovf,
                                    int32_t *ovf_n, int *s_flag, int32_t *s_cnt, Cand *s_top,
                                    int32_t *s_tmp, BigQueue BQ) {
    const uint32_t mask = cap - 1;
    const int32_t i0 = C.ioff[v], deg = C.ioff[v + 1] - i0, nin_v = C.nin[v];
    auto insert_n = [&](int32_t m, unsigned long long qe, uint32_t ninter) {
        uint32_t h = hslot(m, mask);
        for (uint32_t probe = 0; probe < cap; probe++) {
            int32_t k = ((volatile int32_t *)keys)[h];
            if (k == -1) {
                int32_t old = atomicCAS(&keys[h], -1, m);
                if (old == -1) {
                    const uint32_t slot = (uint32_t)atomicAdd(s_cnt, 1);
                    if (slot < limit) slots[slot] = (int32_t)h;
                    else *(volatile int *)s_flag = 1;
                    k = m;
                } else {
                    k = old;
                }
            }
            if (k == m) {
                add_u64_split(&eta[h], qe);
                if (ninter) atomicAdd(&inter[h], ninter);
                return;
            }
            h = (h + 1) & mask;
        }
    };
    cta_walk(C, v, i0, deg, nin_v, s_flag, BQ, insert_n);
    __syncthreads();
    const int overflow = *s_flag;
    const uint64_t capn = *C.cap;
    if (overflow) {
        // the slot list is incomplete: clear the whole table, redo the node in a larger one
        for (uint32_t h = threadIdx.x; h < cap; h += blockDim.x) {
            keys[h] = -1;
            eta[h] = 0;
            inter[h] = 0;
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
    // only the occupied slots, from the slot list
    const int32_t used = *(volatile int32_t *)s_cnt;
    if constexpr (PIMAX <= EMIT_W) {
        TopList<PIMAX> tl;
        tl.init();
        for (int32_t i = threadIdx.x; i < used; i += blockDim.x) {
            const int32_t h = slots[i];
            const int32_t m = keys[h];
            if (pair_valid(C, v, m, (int32_t)inter[h])) tl.push(Cand{eta[h] + pair_noise(C.level_key, v, m, capn), m});
            keys[h] = -1;
            eta[h] = 0;
            inter[h] = 0;
        }
        int32_t tot = used;
        __syncthreads();
        if (threadIdx.x == 0) {
            C.nbcnt[v] = tot;
            *s_cnt = 0;
        }
        block_emit_top<PIMAX>(tl, C, v, s_top);
    } else {
        // rounds of four over the slot list, each below the last entry of the round before
        // (the first round stores the noised scores in eta and the validity
        // in inter)
        Cand thr{~0ull, INT32_MAX};
        for (int r0 = 0; r0 < C.pi; r0 += EMIT_W) {
            TopList<EMIT_W> tl;
            tl.init();
            for (int32_t i = threadIdx.x; i < used; i += blockDim.x) {
                const int32_t h = slots[i];
                const int32_t m = keys[h];
                unsigned long long sc = eta[h];
                bool ok = inter[h] != 0;
                if (r0 == 0) {
                    ok = pair_valid(C, v, m, (int32_t)inter[h]);
                    if (ok) sc += pair_noise(C.level_key, v, m, capn);
                    eta[h] = sc;
                    inter[h] = ok ? 1u : 0u;
                }
                if (ok) {
                    const Cand c{sc, m};
                    if (cand_gt(thr, c)) tl.push(c);
                }
            }
            thr = block_emit_range(tl, C, v, s_top, r0, min(EMIT_W, C.pi - r0), &s_top[32 * PIMAX - 1]);
        }
        for (int32_t i = threadIdx.x; i < used; i += blockDim.x) {
            const int32_t h = slots[i];
            keys[h] = -1;
            eta[h] = 0;
            inter[h] = 0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            C.nbcnt[v] = used;
            *s_cnt = 0;
        }
        __syncthreads();
    }
}

template <int PIMAX, int BT>
__global__ void __launch_bounds__(BT) k_propose_smem(PropCtx C, const int32_t *list, const int32_t *count_p,
                                                     uint32_t cap, uint32_t limit, int32_t *ovf, int32_t *ovf_n) {
    HP_KERNEL_ENTER();
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long *eta = reinterpret_cast<unsigned long long *>(smem);
    uint32_t *inter = reinterpret_cast<uint32_t *>(eta + cap);
    int32_t *keys = reinterpret_cast<int32_t *>(inter + cap);
    int32_t *slots = keys + cap;
    __shared__ Cand s_top[32 * PIMAX];
    __shared__ int32_t s_qe[BT];
    __shared__ unsigned long long s_qq[BT];
    __shared__ uint32_t s_qc[BT];
    __shared__ int32_t s_nbig;
    __shared__ int32_t s_tmp[32];
    __shared__ int s_flag;
    __shared__ int32_t s_cnt;
    const int32_t count = *count_p;
    if (count == 0) return;
    for (uint32_t i = threadIdx.x; i < cap; i += BT) {
        keys[i] = -1;
        eta[i] = 0;
        inter[i] = 0;
    }
    if (threadIdx.x == 0) {
        s_flag = 0;
        s_cnt = 0;
        s_nbig = 0;
    }
    __syncthreads();
    for (int32_t k = blockIdx.x; k < count; k += gridDim.x)
        propose_hashed_node<PIMAX>(C, list[k], keys, eta, inter, cap, limit, slots, ovf, ovf_n, &s_flag, &s_cnt,
                                   s_top, s_tmp, BigQueue{s_qe, s_qq, s_qc, &s_nbig});
}

// one CTA region of gcap slots in global memory per CTA (clean on entry and
// left clean); gcap >= 2 * (nodes of the level) so no node overflows it
template <int PIMAX>
__global__ void __launch_bounds__(PT) k_propose_global(PropCtx C, const int32_t *list, const int32_t *count_p,
                                                       uint32_t gcap, int32_t *gkeys, unsigned long long *geta,
                                                       uint32_t *ginter, int32_t *gslots, int32_t *err_list,
                                                       int32_t *err_n) {
    HP_KERNEL_ENTER();
    __shared__ Cand s_top[32 * PIMAX];
    __shared__ int32_t s_qe[PT];
    __shared__ unsigned long long s_qq[PT];
    __shared__ uint32_t s_qc[PT];
    __shared__ int32_t s_nbig;
    __shared__ int32_t s_tmp[32];
    __shared__ int s_flag;
    __shared__ int32_t s_cnt;
    const int32_t count = *count_p;
    if (count == 0) return;
    const int64_t o = (int64_t)blockIdx.x * gcap;
    if (threadIdx.x == 0) {
        s_flag = 0;
        s_cnt = 0;
        s_nbig = 0;
    }
    __syncthreads();
    for (int32_t k = blockIdx.x; k < count; k += gridDim.x)
        propose_hashed_node<PIMAX>(C, list[k], gkeys + o, geta + o, ginter + o, gcap, gcap - 1, gslots + o, err_list,
                                   err_n, &s_flag, &s_cnt, s_top, s_tmp, BigQueue{s_qe, s_qq, s_qc, &s_nbig});
}

// ---------------------------------------------------------------- node tiers
// warp tier: small neighbourhood bound and little traversal work; hub
// tier: traversals (pin visits or incidence entries) large enough to keep a
// 1024-thread CTA busy
// dense tier (level of at most DENSE_N nodes): neighbourhood bound above
// dense_bound; the others use hashed tables
constexpr long long WARP_VISITS = 4096, HUB_VISITS = 262144;
constexpr int32_t HUB_INCIDENCE = 4096;   // incidence entries: chunks of a 512-thread walk
__global__ void k_tiers(const int32_t *bound, const long long *vis, const int32_t *ioff, int32_t n,
                        uint32_t warp_limit, int32_t dense_bound, int32_t *lW, int32_t *lB, int32_t *lH, int32_t *lD,
                        int32_t *lDH, int32_t *cnt, int32_t pi, int32_t *cand, uint64_t *cscore) {
    HP_KERNEL_ENTER();
    GRID_STRIDE(v, (int64_t)n) {
        if (bound[v] == 0) {
            // no (size-valid) neighbour: an empty candidate list, no walk
            for (int32_t r = 0; r < pi; r++) {
                cand[v * (int64_t)pi + r] = -1;
                cscore[v * (int64_t)pi + r] = 0;
            }
            continue;
        }
        const bool hub = vis[v] > HUB_VISITS || ioff[v + 1] - ioff[v] > HUB_INCIDENCE;
        if ((uint32_t)bound[v] <= warp_limit && vis[v] <= WARP_VISITS) lW[atomicAdd(&cnt[0], 1)] = (int32_t)v;
        else if (bound[v] > dense_bound) {
            if (hub) lDH[atomicAdd(&cnt[7], 1)] = (int32_t)v;
            else lD[atomicAdd(&cnt[6], 1)] = (int32_t)v;
        } else if (hub) lH[atomicAdd(&cnt[5], 1)] = (int32_t)v;
        else lB[atomicAdd(&cnt[1], 1)] = (int32_t)v;
    }
}

// Per-call coarsening workspace (sized for level 0, reused by every level).
struct CoarsenWs {
    int32_t cn, ce, pi;
    uint64_t *q;
    int32_t *canon;   // destination-list groups of the current level's hyperedges
    cudaStream_t side[3] = {nullptr, nullptr, nullptr};   // side streams of the proposal tiers
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    int32_t *cand;      // [n*K] top-K lists of the proposal (K = learned_k, else Pi)
    uint64_t *cscore;
    // learned merge priority (learned_k > 0)
    hp_merge_model *model = nullptr;
    uint8_t *feat = nullptr;
    int32_t *rank = nullptr, *lscore = nullptr, *lcand = nullptr;
    uint64_t *lcs = nullptr;
    int32_t *lW, *lB, *lC, *lG, *lH, *lD, *lDH, *cnt;   // cnt: 0 W 1 B 2 C 3 G 4 errors 5 H 6 D 7 DH
    long long *nsum, *vis;             // per node: sum of (|e|-1), sum of |e| over I(v)
    uint32_t gcap;
    int gnb;
    int32_t *gkeys;
    unsigned long long *geta;
    uint32_t *ginter;
    int32_t *gslots;
    // best-effort pairing and matching
    int32_t *flag, *pos, *target, *ccount, *fillpos, *best;
    uint32_t *ikeys, *iids;
    uint64_t *score;
    long long *ss0, *ss10, *sum0, *kmax;
    LevelBox *box;
};

template <int PIMAX>
static void run_proposal(const PropCtx &C, Level &L, const Params &P, CoarsenWs &W, Arena &A) {
    cudaStream_t s = A.stream();
    const int sms = num_sms();
    const int32_t dbg = P.o.debug_table_cap;
    const uint32_t wcap = dbg > 0 ? std::min<uint32_t>(512, (uint32_t)dbg) : 512;
    uint32_t capB = 4096, capC = 8192;
    if (dbg > 0) capB = capC = (uint32_t)dbg;
    // dense tables only on small levels, for neighbourhoods too large for the first hashed table
    const int32_t dense_bound = (C.n <= DENSE_N && dbg == 0) ? (int32_t)(capB / 2) : 0x7fffffff;
    launch_k(k_tiers, grid_of(C.n, 256), 256, 0, s, L.nbnd, W.vis, L.ioff, C.n, wcap / 2, dense_bound, W.lW, W.lB, W.lH,
                                              W.lD, W.lDH, W.cnt, C.pi, C.cand, C.cscore);
    HP_LAUNCH_CHECK();
    // the tiers take disjoint node lists, so they run side by side: the warp
    // tier, the dense tier and the hub tier each on a side stream, tier B on
    // the main one; tier C (overflows of B and the hubs) waits for the hubs,
    // and the global tier (whose error list reuses the warp list) for all
    cudaStream_t sw = W.side[0], sd = W.side[1], sh = W.side[2];
    HPC(cudaEventRecord(W.ev[0], s));
    for (cudaStream_t x : {sw, sd, sh}) HPC(cudaStreamWaitEvent(x, W.ev[0], 0));
    {
        size_t sm = (size_t)wcap * 16 * (WP_T / 32);
        int occ = prepare_kernel((const void *)k_propose_warp<PIMAX>, WP_T, sm);
        int grid = (int)std::min<int64_t>(cdiv(C.n, WP_T / 32), (int64_t)sms * occ);
        launch_k(k_propose_warp<PIMAX>, std::max(grid, 1), WP_T, sm, sw, C, W.lW, W.cnt + 0, wcap);
        HP_LAUNCH_CHECK();
    }
    if (dense_bound != 0x7fffffff) {
        size_t sm = (size_t)C.n * 12;
        int occ = prepare_kernel((const void *)k_propose_dense<PIMAX, PT>, PT, sm);
        launch_k(k_propose_dense<PIMAX, PT>, std::max(1, std::min<int>(C.n, sms * occ)), PT, sm, sd, C, W.lD, W.cnt + 6);
        HP_LAUNCH_CHECK();
        prepare_kernel((const void *)k_propose_dense<PIMAX, 1024>, 1024, sm);
        launch_k(k_propose_dense<PIMAX, 1024>, sms, 1024, sm, sd, C, W.lDH, W.cnt + 7);
        HP_LAUNCH_CHECK();
    }
    auto smem_of = [](uint32_t cap) { return (size_t)cap * 16 + (size_t)(cap * 3 / 4) * 4; };
    {
        size_t sm = smem_of(capB);
        prepare_kernel((const void *)k_propose_smem<PIMAX, 1024>, 1024, sm);
        launch_k(k_propose_smem<PIMAX, 1024>, sms, 1024, sm, sh, C, W.lH, W.cnt + 5, capB, capB * 3 / 4, W.lC, W.cnt + 2);
        HP_LAUNCH_CHECK();
        int occ = prepare_kernel((const void *)k_propose_smem<PIMAX, 512>, 512, sm);
        launch_k(k_propose_smem<PIMAX, 512>, std::max(1, std::min<int>(C.n, sms * occ)), 512, sm, s,
            C, W.lB, W.cnt + 1, capB, capB * 3 / 4, W.lC, W.cnt + 2);
        HP_LAUNCH_CHECK();
    }
    HPC(cudaEventRecord(W.ev[3], sh));
    HPC(cudaStreamWaitEvent(s, W.ev[3], 0));
    {
        // nodes whose neighbourhood outgrew the first table (the bound can be far above the truth)
        size_t sm = smem_of(capC);
        int occ = prepare_kernel((const void *)k_propose_smem<PIMAX, PT>, PT, sm);
        launch_k(k_propose_smem<PIMAX, PT>, std::max(1, std::min<int>(C.n, sms * occ)), PT, sm, s,
            C, W.lC, W.cnt + 2, capC, capC * 3 / 4, W.lG, W.cnt + 3);
        HP_LAUNCH_CHECK();
    }
    HPC(cudaEventRecord(W.ev[1], sw));
    HPC(cudaEventRecord(W.ev[2], sd));
    HPC(cudaStreamWaitEvent(s, W.ev[1], 0));
    HPC(cudaStreamWaitEvent(s, W.ev[2], 0));
    launch_k(k_propose_global<PIMAX>, W.gnb, PT, 0, s, C, W.lG, W.cnt + 3, W.gcap, W.gkeys, W.geta, W.ginter, W.gslots,
                                                  W.lW, W.cnt + 4);
    HP_LAUNCH_CHECK();
}

// ---------------------------------------------------------------- best-effort pairing
// Each step is a strided loop (t0, nt): a kernel runs it over its grid, the
// one-cluster matching kernel over its cluster, with a barrier in between.
#define CSTRIDE(i, n, t0, nt) for (int64_t i = (t0); i < (int64_t)(n); i += (nt))
#define K_T0 (blockIdx.x * (int64_t)blockDim.x + threadIdx.x)
#define K_NT ((int64_t)gridDim.x * blockDim.x)

__device__ __forceinline__ void ph_iso_flags(const int32_t *cand, int32_t pi, int32_t n, int32_t *flag, int64_t t0,
                                             int64_t nt) {
    CSTRIDE(v, n, t0, nt) flag[v] = cand[(int64_t)v * pi] < 0 ? 1 : 0;
}
__device__ __forceinline__ void ph_iso_compact(const int32_t *flag, const int32_t *pos, const int32_t *size,
                                               int32_t n, uint32_t *keys, uint32_t *vals, int64_t t0, int64_t nt) {
    CSTRIDE(v, n, t0, nt) {
        if (flag[v]) {
            keys[pos[v]] = (uint32_t)size[v];
            vals[pos[v]] = (uint32_t)v;
        }
    }
}
__device__ __forceinline__ void ph_iso_pair(const uint32_t *ids, int32_t k, const int32_t *size, const int32_t *nin,
                                            int32_t omega, int32_t delta, int32_t *mate, unsigned long long *pairs,
                                            int64_t t0, int64_t nt) {
    CSTRIDE(i, k / 2, t0, nt) {
        int32_t a = (int32_t)ids[i], b = (int32_t)ids[k - 1 - i];
        if ((int64_t)size[a] + size[b] <= omega && (int64_t)nin[a] + nin[b] <= delta) {
            mate[a] = b;
            mate[b] = a;
            atomicAdd(pairs, 1ull);
        }
    }
}
__global__ void k_iso_flags(const int32_t *cand, int32_t pi, int32_t n, int32_t *flag) {
    HP_KERNEL_ENTER();
    ph_iso_flags(cand, pi, n, flag, K_T0, K_NT);
}
__global__ void k_iso_compact(const int32_t *flag, const int32_t *pos, const int32_t *size, int32_t n, uint32_t *keys,
                              uint32_t *vals) {
    HP_KERNEL_ENTER();
    ph_iso_compact(flag, pos, size, n, keys, vals, K_T0, K_NT);
}
__global__ void k_iso_pair(const uint32_t *ids, const int32_t *cntp, const int32_t *size, const int32_t *nin,
                           int32_t omega, int32_t delta, int32_t *mate, unsigned long long *pairs) {
    HP_KERNEL_ENTER();
    ph_iso_pair(ids, *cntp, size, nin, omega, delta, mate, pairs, K_T0, K_NT);
}

// ---------------------------------------------------------------- matching
__device__ __forceinline__ void ph_targets(const int32_t *cand, const uint64_t *cscore, int32_t pi,
                                           const int32_t *mate, int32_t n, int32_t *target, uint64_t *score,
                                           long long *sum0, long long *kmax, int32_t *best, int32_t *ccount,
                                           int32_t *pending, int64_t t0, int64_t nt) {
    CSTRIDE(v, n, t0, nt) {
        sum0[v] = 0;
        kmax[v] = LLONG_MIN;
        best[v] = -1;
        ccount[v] = 0;
        pending[v] = 0;
        int32_t t = -1;
        uint64_t sc = 0;
        if (mate[v] < 0) {
            for (int32_t i = 0; i < pi; i++) {
                int32_t c = cand[(int64_t)v * pi + i];
                if (c < 0) break;
                if (mate[c] < 0) {
                    t = c;
                    sc = cscore[(int64_t)v * pi + i];
                    break;
                }
            }
        }
        target[v] = t;
        score[v] = sc;
    }
}

// |child(n) \ R| per node, twice: the count and the counter of children still to finish
__device__ __forceinline__ void ph_child_count(const int32_t *target, int32_t n, int32_t *ccount, int32_t *pending,
                                               int64_t t0, int64_t nt) {
    const int lane = threadIdx.x & 31;
    CSTRIDE(v, n, t0, nt) {
        // the lanes of a warp with the same parent count once (stars)
        const unsigned act = __activemask();
        const int32_t t = target[v];
        const bool child = t >= 0 && target[t] != v;
        const unsigned g = __match_any_sync(act, child ? t : -1 - lane);
        if (child && (g & ((1u << lane) - 1u)) == 0u) {
            atomicAdd(&ccount[t], __popc(g));
            atomicAdd(&pending[t], __popc(g));
        }
    }
}

__global__ void k_targets(const int32_t *cand, const uint64_t *cscore, int32_t pi, const int32_t *mate, int32_t n,
                          int32_t *target, uint64_t *score, long long *sum0, long long *kmax, int32_t *best,
                          int32_t *ccount, int32_t *pending) {
    HP_KERNEL_ENTER();
    ph_targets(cand, cscore, pi, mate, n, target, score, sum0, kmax, best, ccount, pending, K_T0, K_NT);
}
__global__ void k_child_count(const int32_t *target, int32_t n, int32_t *ccount, int32_t *pending) {
    HP_KERNEL_ENTER();
    ph_child_count(target, n, ccount, pending, K_T0, K_NT);
}

struct DpCtx {
    int32_t n;
    const int32_t *target, *ccount;   // ccount: |child(n) \ R|
    const uint64_t *score;
    int32_t *pending;                 // children still to finish
    long long *ss0, *ss10;
    long long *sum0;                  // sum of the children's ss0 (accumulated by them)
    long long *kmax;                  // max of the children's ss1-0 (accumulated by them)
    int32_t *best;
    uint32_t *err;
    uint32_t *level_err;              // the level's error word, read by the host before contraction
    int32_t walk_cap;                 // steps a walk may take (n, or less in the bounded-loop test)
};
__device__ __forceinline__ void dp_timeout(const DpCtx &D) {
    atomicOr(D.err, E_TIMEOUT);
    atomicOr(D.level_err, E_TIMEOUT);
}

// Bottom-up (Eq. 7, 8, 10): a thread starts at every leaf and climbs.  A
// finished child adds its ss0 to the parent's sum0 and raises the parent's
// kmax to its ss1-0, then counts itself off; the thread finishing the last
// child continues with the parent, whose children are then all accounted
// for, so no node's children are ever walked one by one.  A parent with a
// single child takes the child's values from registers (plain stores, no
// fence, no counter).  The best child itself (largest ss1-0, ties to the
// larger id) is found afterwards by k_best_child.
__device__ __forceinline__ void ph_dp_up(const DpCtx &D, int64_t t0, int64_t nt) {
    const int lane = threadIdx.x & 31;
    CSTRIDE(v0, D.n, t0, nt) {
        const unsigned act = __activemask();
        const int32_t v = (int32_t)v0;
        const bool leaf = D.ccount[v] == 0 && D.target[v] >= 0;   // a leaf with a proposal edge
        const int32_t tv = leaf ? D.target[v] : -1;
        const bool multi = leaf && D.target[tv] != v && D.ccount[tv] > 1;
        // Leaves whose parent has several children take their first step with
        // the warp's other leaves of that parent: a leaf's ss0 is 0, so it adds
        // nothing to the parent's sum0; each raises kmax (a load first: most
        // are below it); one counter update per group, and the group that
        // finishes the parent's children climbs on from it.  Star-shaped
        // proposal graphs (a hub with a thousand leaves) then cost a few
        // atomics per warp instead of three per leaf.
        const unsigned g = __match_any_sync(act, multi ? tv : -1 - lane);
        int32_t cur = v, steps0 = 0;
        if (multi) {
            const long long my10 = (long long)D.score[v];
            __stcg(&D.ss0[v], 0ll);
            __stcg(&D.ss10[v], my10);
            if (my10 > __ldcg(&D.kmax[tv])) atomicMax(&D.kmax[tv], my10);
            __syncwarp(g);
            bool last = false;
            if ((g & ((1u << lane) - 1u)) == 0u) {
                __threadfence();
                last = atomicSub(&D.pending[tv], (int)__popc(g)) == (int)__popc(g);
                __threadfence();
            }
            if (!last) continue;
            cur = tv;
            steps0 = 1;
        } else if (!leaf) {
            continue;
        }
        bool carried = false;                       // cur's single child's values in registers
        long long cs0 = 0, cmax = 0;
        for (int32_t steps = steps0;; steps++) {
            if (steps > D.walk_cap) {
                dp_timeout(D);
                break;
            }
            const int32_t nk = D.ccount[cur];
            long long s0 = 0, mx = 0;
            if (carried) {
                s0 = cs0;
                mx = cmax;
            } else if (nk > 0) {
                s0 = __ldcg(&D.sum0[cur]);
                mx = __ldcg(&D.kmax[cur]);
            }
            const long long my0 = s0 + ((nk > 0 && mx > 0) ? mx : 0);
            __stcg(&D.ss0[cur], my0);
            const int32_t t = D.target[cur];
            if (t < 0 || D.target[t] == cur) break;   // a root
            const long long my10 = (long long)D.score[cur] + s0 - my0;
            __stcg(&D.ss10[cur], my10);
            if (D.ccount[t] == 1) {
                __stcg(&D.sum0[t], my0);
                __stcg(&D.kmax[t], my10);
                carried = true;
                cs0 = my0;
                cmax = my10;
            } else {
                atomicAdd((unsigned long long *)&D.sum0[t], (unsigned long long)my0);
                atomicMax(&D.kmax[t], my10);
                __threadfence();
                if (atomicSub(&D.pending[t], 1) != 1) break;
                __threadfence();
                carried = false;
            }
            cur = t;
        }
    }
}

// best(t) = the child of t (partner root excluded) with the largest ss1-0,
// ties to the larger id
__device__ __forceinline__ void ph_best_child(const DpCtx &D, int64_t t0, int64_t nt) {
    CSTRIDE(v0, D.n, t0, nt) {
        const int32_t v = (int32_t)v0, t = D.target[v];
        if (t >= 0 && D.target[t] != v && __ldcg(&D.ss10[v]) == __ldcg(&D.kmax[t])) atomicMax(&D.best[t], v);
    }
}

// Top-down (Eq. 11, 12): up(v) = v matched to target(v).  A node is up iff
// it is its parent's best child with ss1-0 > 0 and the parent is not up; the
// chain of such links ends at a node that is not up or at a root.
__device__ __forceinline__ void ph_dp_down(const DpCtx &D, const int32_t *target, int32_t *mate,
                                           unsigned long long *pairs, int64_t t0, int64_t nt) {
    CSTRIDE(v0, D.n, t0, nt) {
        int32_t v = (int32_t)v0;
        if (target[v] < 0) continue;
        int32_t cur = v, k = 0;
        bool base = false;
        for (int32_t steps = 0;; steps++) {
            if (steps > D.walk_cap) {
                dp_timeout(D);
                break;
            }
            int32_t t = target[cur];
            if (t < 0) {
                base = false;
                break;
            }
            if (target[t] == cur) {
                long long ss1 = (long long)D.score[cur] + __ldcg(&D.sum0[cur]) + __ldcg(&D.sum0[t]);
                base = ss1 > __ldcg(&D.ss0[cur]) + __ldcg(&D.ss0[t]);
                break;
            }
            if (D.best[t] != cur || __ldcg(&D.ss10[cur]) <= 0) {
                base = false;
                break;
            }
            cur = t;
            k++;
        }
        bool up = base ^ (k & 1);
        if (up) {
            int32_t t = target[v];
            mate[v] = t;
            mate[t] = v;
            if (target[t] != v || v < t) atomicAdd(pairs, 1ull);
        }
    }
}

// In-degree of every node in the first proposal graph (its non-root children
// plus its 2-cycle partner): the number of distinct targets and the largest
// in-degree go to the level's box (a diagnostic of the pairing).
__device__ __forceinline__ void ph_indeg(const int32_t *target, const int32_t *ccount, int32_t n, LevelBox *box,
                                         int64_t t0, int64_t nt) {
    int32_t mx = 0, cnt = 0;
    CSTRIDE(v, n, t0, nt) {
        const int32_t t = target[v];
        const int32_t d = ccount[v] + ((t >= 0 && target[t] == (int32_t)v) ? 1 : 0);
        mx = max(mx, d);
        cnt += d > 0 ? 1 : 0;
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
        cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (mx) atomicMax(&box->maxin, mx);
        if (cnt) atomicAdd(&box->ntargets, cnt);
    }
}
__global__ void k_indeg(const int32_t *target, const int32_t *ccount, int32_t n, LevelBox *box) {
    HP_KERNEL_ENTER();
    ph_indeg(target, ccount, n, box, K_T0, K_NT);
}
__global__ void k_dp_up(DpCtx D) { HP_KERNEL_ENTER(); ph_dp_up(D, K_T0, K_NT); }
__global__ void k_best_child(DpCtx D) { HP_KERNEL_ENTER(); ph_best_child(D, K_T0, K_NT); }
__global__ void k_dp_down(DpCtx D, const int32_t *target, int32_t *mate, unsigned long long *pairs) {
    HP_KERNEL_ENTER();
    ph_dp_down(D, target, mate, pairs, K_T0, K_NT);
}

// ---------------------------------------------------------------- one-cluster matching
// The best-effort pairing and the pi matching rounds of a level of at most
// sq_max<uint32_t>() nodes in one launch: the steps of the multi-kernel form, each a
// strided loop over the cluster's threads, separated by cluster barriers.
struct MatchArgs {
    const int32_t *candK;   // proposal lists (K entries): nodes without a valid neighbour
    int32_t K;
    const int32_t *cand;    // C(n) and its weights (pi entries)
    const uint64_t *cscore;
    int32_t pi, n, omega, delta;
    const int32_t *size, *nin;
    int32_t *flag, *pos;
    uint32_t *ikeys, *iids;
    int32_t isobits;
    int32_t *mate;
    LevelBox *box;
    int32_t *target, *ccount;   // the writable views of D's arrays
    uint64_t *score;
    DpCtx D;
};
__global__ void __cluster_dims__(SQ_CS, 1, 1) __launch_bounds__(SQ_T) k_match_cluster(MatchArgs A) {
    HP_KERNEL_ENTER();
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_wc[32 * 256];
    __shared__ uint32_t s_tot[256];
    __shared__ uint32_t s_base[512];
    __shared__ int32_t s_tmp[40];
    __shared__ int32_t s_part;
    cg::cluster_group cl = cg::this_cluster();
    const int64_t t0 = (int64_t)cl.block_rank() * blockDim.x + threadIdx.x, nt = (int64_t)SQ_CS * blockDim.x;
    const SqBuf<uint32_t> B(smem);
    const int32_t n = A.n;
    // best-effort pairing (Sec. V-C): nodes with no valid neighbour, by (size, id)
    ph_iso_flags(A.candK, A.K, n, A.flag, t0, nt);
    cl.sync();
    const int32_t k = cluster_scan_excl<int32_t>(cl, A.flag, A.pos, n, s_tmp, &s_part);
    if (t0 == 0) A.box->isolist = k;
    ph_iso_compact(A.flag, A.pos, A.size, n, A.ikeys, A.iids, t0, nt);
    cl.sync();
    cluster_radix_sort<uint32_t>(cl, A.ikeys, A.iids, k, (A.isobits + 7) / 8, B, s_wc, s_tot, s_base);
    ph_iso_pair(A.iids, k, A.size, A.nin, A.omega, A.delta, A.mate, &A.box->iso, t0, nt);
    cl.sync();
    // pi rounds of maximum-weight matching (Sec. V-D)
    const DpCtx &D = A.D;
    unsigned long long before = 0;   // pairs before the round
    for (int32_t r = 0; r < A.pi; r++) {
        ph_targets(A.cand, A.cscore, A.pi, A.mate, n, A.target, A.score, D.sum0, D.kmax, D.best, A.ccount, D.pending,
                   t0, nt);
        cl.sync();
        ph_child_count(A.target, n, A.ccount, D.pending, t0, nt);
        cl.sync();
        if (r == 0) ph_indeg(A.target, A.ccount, n, A.box, t0, nt);
        ph_dp_up(D, t0, nt);
        cl.sync();
        ph_best_child(D, t0, nt);
        cl.sync();
        ph_dp_down(D, D.target, A.mate, &A.box->pairs, t0, nt);
        cl.sync();
        if (r == 0 && t0 == 0) A.box->pairs1 = A.box->pairs;
        // a round that forms no pair leaves every target as it was, so every
        // later round would form none either
        const unsigned long long after = *(volatile unsigned long long *)&A.box->pairs;
        if (after == before) break;
        before = after;   // (the count changes again only after two more cluster barriers)
    }
}

__global__ void k_sum_i32(const int32_t *x, int32_t n, unsigned long long *sum) {
    HP_KERNEL_ENTER();
    unsigned long long loc = 0;
    GRID_STRIDE(i, (int64_t)n) loc += (unsigned long long)x[i];
    for (int o = 16; o > 0; o >>= 1) loc += __shfl_down_sync(0xffffffffu, loc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(sum, loc);
}
__global__ void k_flag_if_nonzero(const int32_t *x, uint32_t *err) {
    HP_KERNEL_ENTER();
    if (*x) atomicOr(err, E_INTERNAL);
}

static CoarsenWs *coarsen_workspace_body(CoarsenWs *W, int32_t n, int32_t e, const Params &P, Arena &A);

// on a failure half-way, the streams and events made so far are destroyed
// (the arena frees the device memory taken so far)
CoarsenWs *coarsen_workspace(int32_t n, int32_t e, const Params &P, Arena &A) {
    CoarsenWs *W = new CoarsenWs();
    try {
        return coarsen_workspace_body(W, n, e, P, A);
    } catch (...) {
        for (cudaStream_t x : W->side)
            if (x) cudaStreamDestroy(x);
        for (cudaEvent_t x : W->ev)
            if (x) cudaEventDestroy(x);
        delete W;
        throw;
    }
}

static CoarsenWs *coarsen_workspace_body(CoarsenWs *W, int32_t n, int32_t e, const Params &P, Arena &A) {
    cudaStream_t s = A.stream();
    for (cudaStream_t &x : W->side) HPC(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
    for (cudaEvent_t &x : W->ev) HPC(cudaEventCreateWithFlags(&x, cudaEventDisableTiming));
    const int32_t pi = P.o.pi, K = P.o.learned_k > 0 ? P.o.learned_k : pi;
    W->cn = n;
    W->ce = e;
    W->pi = pi;
    W->q = A.get<uint64_t>(e);
    W->canon = A.get<int32_t>(std::max(e, 1) + 1);   // + the flag of dst_groups_of
    W->cand = A.get<int32_t>((int64_t)n * K);
    W->cscore = A.get<uint64_t>((int64_t)n * K);
    if (P.o.learned_k > 0) {
        // no model: the workspace of the feature extraction alone
        if (P.o.merge_model) {
            W->model = A.get<hp_merge_model>(1);
            HPC(cudaMemcpyAsync(W->model, P.o.merge_model, sizeof(hp_merge_model), cudaMemcpyHostToDevice, s));
        }
        // per-pair rows of one pass of node_batch nodes (all nodes without it)
        const int64_t rows = (int64_t)(P.o.node_batch > 0 ? std::min(P.o.node_batch, std::max(n, 1)) : n) * K;
        W->feat = A.get<uint8_t>(rows * 16);
        W->rank = A.get<int32_t>(rows);
        W->lscore = A.get<int32_t>(rows);
        W->lcand = A.get<int32_t>((int64_t)n * pi);
        W->lcs = A.get<uint64_t>((int64_t)n * pi);
    }
    W->lW = A.get<int32_t>(n);
    W->lB = A.get<int32_t>(n);
    W->lC = A.get<int32_t>(n);
    W->lG = A.get<int32_t>(n);
    W->lH = A.get<int32_t>(n);
    W->lD = A.get<int32_t>(n);
    W->lDH = A.get<int32_t>(n);
    W->cnt = A.get<int32_t>(8);
    W->nsum = A.get<long long>(n);
    W->vis = A.get<long long>(n);
    // global neighbour tables: one region of gcap >= 2n slots per CTA
    W->gcap = 64;
    while (W->gcap < 2u * (uint32_t)std::max(n, 1) + 2u && W->gcap < (1u << 30)) W->gcap <<= 1;
    W->gnb = (int)std::max<int64_t>(1, std::min<int64_t>(2 * num_sms(), ((int64_t)1 << 28) / ((int64_t)W->gcap * 16)));
    W->gkeys = A.get<int32_t>((int64_t)W->gnb * W->gcap);
    W->geta = A.get<unsigned long long>((int64_t)W->gnb * W->gcap);
    W->ginter = A.get<uint32_t>((int64_t)W->gnb * W->gcap);
    W->gslots = A.get<int32_t>((int64_t)W->gnb * W->gcap);
    HPC(cudaMemsetAsync(W->gkeys, 0xff, sizeof(int32_t) * W->gnb * W->gcap, s));
    HPC(cudaMemsetAsync(W->geta, 0, sizeof(unsigned long long) * W->gnb * W->gcap, s));
    HPC(cudaMemsetAsync(W->ginter, 0, sizeof(uint32_t) * W->gnb * W->gcap, s));
    W->flag = A.get<int32_t>(n);
    W->pos = A.get<int32_t>(n + 1);
    W->ikeys = A.get<uint32_t>(n);
    W->iids = A.get<uint32_t>(n);
    W->target = A.get<int32_t>(n);
    W->score = A.get<uint64_t>(n);
    W->ccount = A.get<int32_t>(n + 1);
    W->fillpos = A.get<int32_t>(n);
    W->best = A.get<int32_t>(n);
    W->ss0 = A.get<long long>(n);
    W->ss10 = A.get<long long>(n);
    W->sum0 = A.get<long long>(n);
    W->kmax = A.get<long long>(n);
    W->box = A.get<LevelBox>(1);
    return W;
}

void coarsen_workspace_free(CoarsenWs *W, Arena &A) {
    if (!W) return;
    // side-stream work must be done before the arena hands its memory back
    // (it is, unless the call is ending early on an error)
    for (cudaStream_t x : W->side)
        if (x) {
            (void)cudaStreamSynchronize(x);
            cudaStreamDestroy(x);
        }
    for (cudaEvent_t x : W->ev)
        if (x) cudaEventDestroy(x);
    for (void *p : {(void *)W->nsum, (void *)W->vis, (void *)W->q, (void *)W->canon, (void *)W->cand, (void *)W->cscore, (void *)W->lW, (void *)W->lB, (void *)W->lC,
                    (void *)W->lG, (void *)W->lH, (void *)W->lD, (void *)W->lDH, (void *)W->cnt, (void *)W->gkeys, (void *)W->geta, (void *)W->ginter, (void *)W->gslots,
                    (void *)W->flag, (void *)W->pos, (void *)W->ikeys, (void *)W->iids, (void *)W->target,
                    (void *)W->score, (void *)W->ccount, (void *)W->fillpos,
                    (void *)W->best, (void *)W->ss0, (void *)W->ss10, (void *)W->sum0, (void *)W->kmax, (void *)W->box})
        A.release(p);
    for (void *p : {(void *)W->model, (void *)W->feat, (void *)W->rank, (void *)W->lscore, (void *)W->lcand,
                    (void *)W->lcs})
        if (p) A.release(p);
    delete W;
}

LevelBox *coarsen_box(CoarsenWs *W) { return W->box; }

// One coarsening level, entirely on the device (no host synchronisation);
// the counters end up in the workspace box.
// on: the groups pay (on average two hyperedges or more per group)
__global__ void k_dst_flag(const int32_t *ngroups, int32_t e, int32_t *on) { HP_KERNEL_ENTER(); *on = 2 * (int64_t)*ngroups <= e; }

// canon[] of the level's hyperedges (see k_dst_hash) and canon_on
static void dst_groups(const Level &L, int32_t *canon, int32_t *canon_on, Arena &A) {
    cudaStream_t s = A.stream();
    const int32_t e = L.e;
    if (e <= 0) return;
    uint32_t *key = A.get<uint32_t>(e), *val = A.get<uint32_t>(e);
    int32_t *nr = A.get<int32_t>(e), *rp = A.get<int32_t>(e + 1), *rep = A.get<int32_t>(e);
    launch_k(k_dst_hash, grid_of((int64_t)e * 32, 256), 256, 0, s, L.off, L.pin, L.nsrc, e, key, val);
    HP_LAUNCH_CHECK();
    radix_sort(key, val, e, 32, A);
    launch_k(k_dst_runs, grid_of((int64_t)e * 32, 256), 256, 0, s, key, val, L.off, L.pin, L.nsrc, e, nr);
    HP_LAUNCH_CHECK();
    scan_excl(nr, rp, e, rp + e, A);
    launch_k(k_dst_rep, grid_of(e, 256), 256, 0, s, val, nr, rp, e, rep);
    HP_LAUNCH_CHECK();
    launch_k(k_dst_canon, grid_of(e, 256), 256, 0, s, val, nr, rp, rep, e, canon);
    HP_LAUNCH_CHECK();
    launch_k(k_dst_flag, 1, 1, 0, s, rp + e, e, canon_on);
    HP_LAUNCH_CHECK();
    for (void *p : {(void *)key, (void *)val, (void *)nr, (void *)rp, (void *)rep}) A.release(p);
}

// The top-K valid neighbours by (eta, id) of every node of the level into
// W.cand / W.cscore (Sec. V-C, Eq. 5-6), and the level's counters into the
// box.  The level must have at least one node.
static void propose_lists(Level &L, int32_t level, const int32_t *w, const Params &P, int32_t K, CoarsenWs &W,
                          Arena &A, cudaEvent_t *prop_events) {
    cudaStream_t s = A.stream();
    const int32_t n = L.n;
    LevelBox *box = W.box;
    static_assert(sizeof(LevelBox) % sizeof(uint32_t) == 0 && sizeof(LevelBox) / sizeof(uint32_t) <= 256,
                  "the level box is zeroed by the first block of k_level_start");
    launch_k(k_level_start, grid_of(std::max<int64_t>(n, 256), 256), 256, 0, s, box, W.nsum, W.vis, n, W.cnt);
    HP_LAUNCH_CHECK();
    if (L.e > 0) {
        launch_k(k_level_q, grid_of(L.e, 256), 256, 0, s, L.off, w, L.e, W.q, &box->qsum);
        HP_LAUNCH_CHECK();
    }
    if (L.np > 0) {
        launch_k(k_node_sums, grid_of(L.np, 256), 256, 0, s, L.off, L.inc, L.inode, L.np, W.nsum, W.vis, &box->visits);
        HP_LAUNCH_CHECK();
    }
    launch_k(k_node_bounds, grid_of(n, 256), 256, 0, s, W.nsum, n, L.nbnd, box, L.e, P.o.noise_permille);
    HP_LAUNCH_CHECK();
    PropCtx C;
    C.n = n;
    C.pi = K;
    C.off = L.off;
    C.pin = L.pin;
    C.nsrc = L.nsrc;
    C.size = L.size;
    C.ioff = L.ioff;
    C.inc = L.inc;
    C.nin = L.nin;
    C.q = W.q;
    C.cap = &box->cap;
    {
        // the level key folds seed and level exactly as the oracle's noise
        uint64_t z = P.seed + 0x9E3779B97F4A7C15ull * (uint64_t)(level + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        C.level_key = z ^ (z >> 31);
    }
    C.omega = P.omega;
    C.delta = P.delta;
    C.cand = W.cand;
    C.cscore = W.cscore;
    C.nbcnt = L.nbnd;   // exact counts replace the bounds (used to size the next level)
    C.canon = nullptr;
    C.canon_on = W.canon + std::max(W.ce, 1);
    // level 0 of a call has unit sizes (every pair passes when Omega >= 2):
    // no filter there, no size gathers
    C.size_filter = level > 0 ? 1 : 0;
    if (prop_events) HPC(cudaEventRecord(prop_events[0], s));   // the grouping counts as proposal time
    if (L.np >= 16 * (int64_t)L.e) {
        // levels of large hyperedges: those with equal destination lists (the
        // channels of one source in a layered network, before and after
        // contraction) are walked once per warp group
        dst_groups(L, W.canon, W.canon + std::max(W.ce, 1), A);
        C.canon = W.canon;
    }
    if (K <= 4) run_proposal<4>(C, L, P, W, A);
    else run_proposal<16>(C, L, P, W, A);
}

// the learned priority's view of a level whose top-K lists are in W
static LearnIn learn_in(const Level &L, int32_t level, const Params &P, int32_t K, CoarsenWs &W) {
    LearnIn X;
    X.n = L.n;
    X.K = K;
    X.pi = P.o.pi;
    X.level = level;
    X.omega = P.omega;
    X.delta = P.delta;
    X.size = L.size;
    X.ioff = L.ioff;
    X.inc = L.inc;
    X.nin = L.nin;
    X.candK = W.cand;
    X.csK = W.cscore;
    X.model = W.model;
    X.feat = W.feat;
    X.rank = W.rank;
    X.score = W.lscore;
    X.cand = W.lcand;
    X.cscore = W.lcs;
    return X;
}

void level_features(Level &L, const int32_t *w, const Params &P, CoarsenWs &W, Arena &A, uint32_t *err_dev,
                    int32_t *cand_out, int32_t *rank_out, uint8_t *feat_out) {
    cudaStream_t s = A.stream();
    const int32_t K = P.o.learned_k;
    if (L.n == 0) return;
    propose_lists(L, 0, w, P, K, W, A, nullptr);
    launch_k(k_flag_if_nonzero, 1, 1, 0, s, W.cnt + 4, err_dev);
    HP_LAUNCH_CHECK();
    LearnIn X = learn_in(L, 0, P, K, W);
    X.feat = feat_out;
    X.rank = rank_out;
    merge_features(X, s);
    HPC(cudaMemcpyAsync(cand_out, W.cand, sizeof(int32_t) * L.n * K, cudaMemcpyDeviceToDevice, s));
}

void coarsen_level(Level &L, int32_t level, const int32_t *w, const Params &P, int32_t *mate, CoarsenWs &W, Arena &A,
                   uint32_t *err_dev, int32_t *cand_out, uint64_t *score_out, cudaEvent_t *prop_events) {
    cudaStream_t s = A.stream();
    const int32_t n = L.n, pi = P.o.pi;
    const bool learned = P.o.learned_k > 0 && (P.o.learned_levels == 0 || level < P.o.learned_levels);
    const int32_t K = learned ? P.o.learned_k : pi;   // length of the proposal's lists
    LevelBox *box = W.box;
    fill_i32(mate, n, -1, s);
    if (n == 0) {
        HPC(cudaMemsetAsync(box, 0, sizeof(LevelBox), s));
        return;
    }
    propose_lists(L, level, w, P, K, W, A, prop_events);
    // C(n) and its matching weights
    int32_t *cand = W.cand;
    uint64_t *cscore = W.cscore;
    if (learned) {
        LearnIn X = learn_in(L, level, P, K, W);
        cand = X.cand;
        cscore = X.cscore;
        learned_candidates(X, P.o.node_batch, s);
    }
    if (prop_events) HPC(cudaEventRecord(prop_events[1], s));
    launch_k(k_flag_if_nonzero, 1, 1, 0, s, W.cnt + 4, err_dev);
    HP_LAUNCH_CHECK();
    launch_k(k_sum_i32, grid_of(n, 256), 256, 0, s, L.nbnd, n, &box->nbrs);
    HP_LAUNCH_CHECK();
    if (cand_out) {
        HPC(cudaMemcpyAsync(cand_out, cand, sizeof(int32_t) * n * pi, cudaMemcpyDeviceToDevice, s));
        HPC(cudaMemcpyAsync(score_out, cscore, sizeof(uint64_t) * n * pi, cudaMemcpyDeviceToDevice, s));
    }

    DpCtx D;
    D.n = n;
    D.target = W.target;
    D.ccount = W.ccount;
    D.score = W.score;
    D.pending = W.fillpos;
    D.ss0 = W.ss0;
    D.ss10 = W.ss10;
    D.sum0 = W.sum0;
    D.kmax = W.kmax;
    D.best = W.best;
    D.err = err_dev;
    D.level_err = &box->err;
    D.walk_cap = P.o.debug_walk_cap > 0 ? std::min(P.o.debug_walk_cap, n) : n;
    if (n <= sq_max<uint32_t>()) {
        // small level: pairing and matching by one cluster, one launch
        MatchArgs M{W.cand, K, cand, cscore, pi, n, P.omega, P.delta, L.size, L.nin, W.flag, W.pos, W.ikeys, W.iids,
                    bits_for((uint64_t)P.omega), mate, box, W.target, W.ccount, W.score, D};
        prepare_kernel((const void *)k_match_cluster, SQ_T, SQ_SMEM);
        launch_k(k_match_cluster, SQ_CS, SQ_T, SQ_SMEM, s, M);
        HP_LAUNCH_CHECK();
        return;
    }

    // best-effort pairing of nodes with no valid neighbour (Sec. V-C)
    launch_k(k_iso_flags, grid_of(n, 256), 256, 0, s, W.cand, K, n, W.flag);
    HP_LAUNCH_CHECK();
    scan_excl(W.flag, W.pos, n, W.pos + n, A);
    HPC(cudaMemcpyAsync(&box->isolist, W.pos + n, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    launch_k(k_iso_compact, grid_of(n, 256), 256, 0, s, W.flag, W.pos, L.size, n, W.ikeys, W.iids);
    HP_LAUNCH_CHECK();
    radix_sort_dev(W.ikeys, W.iids, W.pos + n, n, bits_for((uint64_t)P.omega), A);
    launch_k(k_iso_pair, grid_of(n / 2 + 1, 256), 256, 0, s, W.iids, W.pos + n, L.size, L.nin, P.omega, P.delta, mate,
                                                         &box->iso);
    HP_LAUNCH_CHECK();

    // Pi rounds of maximum-weight matching (Sec. V-D)
    for (int32_t r = 0; r < pi; r++) {
        launch_k(k_targets, grid_of(n, 256), 256, 0, s, cand, cscore, pi, mate, n, W.target, W.score, W.sum0, W.kmax,
                                                  W.best, W.ccount, W.fillpos);
        HP_LAUNCH_CHECK();
        launch_k(k_child_count, grid_of(n, 256), 256, 0, s, W.target, n, W.ccount, W.fillpos);
        HP_LAUNCH_CHECK();
        if (r == 0) {
            launch_k(k_indeg, grid_of(n, 256), 256, 0, s, W.target, W.ccount, n, box);
            HP_LAUNCH_CHECK();
        }
        launch_k(k_dp_up, grid_of(n, 256), 256, 0, s, D);
        HP_LAUNCH_CHECK();
        launch_k(k_best_child, grid_of(n, 256), 256, 0, s, D);
        HP_LAUNCH_CHECK();
        launch_k(k_dp_down, grid_of(n, 256), 256, 0, s, D, W.target, mate, &box->pairs);
        HP_LAUNCH_CHECK();
        if (r == 0)
            HPC(cudaMemcpyAsync(&box->pairs1, &box->pairs, sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s));
    }
}

}  // namespace hp
