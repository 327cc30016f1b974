// hp_cluster.cuh -- CTA- and cluster-wide building blocks of the kernels that
// run one small step on one thread-block cluster: prefix sums, maxima and a
// stable LSD radix sort whose buckets move between the CTAs' shared memory
// (distributed shared memory).  Every thread of every CTA of the cluster
// calls them together.
#pragma once

#include <cooperative_groups.h>

#include <climits>
#include <cstdint>

namespace hp {
namespace cg = cooperative_groups;

__device__ __forceinline__ int32_t block_sum(int32_t x, int32_t *s_tmp) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) s_tmp[threadIdx.x >> 5] = x;
    __syncthreads();
    int32_t t = 0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < (blockDim.x >> 5) ? s_tmp[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) s_tmp[32] = t;
    }
    __syncthreads();
    t = s_tmp[32];
    __syncthreads();
    return t;
}
// exclusive prefix sum of in[0..n) into out, by one CTA
__device__ __forceinline__ void block_scan_excl(const int32_t *in, int32_t *out, int64_t n, int32_t *s_tmp) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int32_t carry = 0;
    for (int64_t base = 0; base < n; base += blockDim.x) {
        int64_t i = base + threadIdx.x;
        int32_t x = i < n ? in[i] : 0, inc = x;
        for (int o = 1; o < 32; o <<= 1) {
            int32_t u = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += u;
        }
        if (lane == 31) s_tmp[wid] = inc;
        __syncthreads();
        if (wid == 0) {
            int32_t y = lane < nw ? s_tmp[lane] : 0, yi = y;
            for (int o = 1; o < 32; o <<= 1) {
                int32_t u = __shfl_up_sync(0xffffffffu, yi, o);
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

// sum over the CTA (all threads take part; s_ll holds 33 words)
__device__ __forceinline__ long long block_sum_ll(long long x, long long *s_ll) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) s_ll[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
        long long y = threadIdx.x < (blockDim.x >> 5) ? s_ll[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) y += __shfl_down_sync(0xffffffffu, y, o);
        if (threadIdx.x == 0) s_ll[32] = y;
    }
    __syncthreads();
    const long long r = s_ll[32];
    __syncthreads();
    return r;
}

// maximum over the CTA (all threads take part; s_ll holds 33 words)
__device__ __forceinline__ long long block_max_ll(long long x, long long *s_ll) {
    for (int o = 16; o > 0; o >>= 1) x = max(x, __shfl_xor_sync(0xffffffffu, x, o));
    if ((threadIdx.x & 31) == 0) s_ll[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
        long long y = threadIdx.x < (blockDim.x >> 5) ? s_ll[threadIdx.x] : LLONG_MIN;
        for (int o = 16; o > 0; o >>= 1) y = max(y, __shfl_xor_sync(0xffffffffu, y, o));
        if (threadIdx.x == 0) s_ll[32] = y;
    }
    __syncthreads();
    const long long r = s_ll[32];
    __syncthreads();
    return r;
}
__device__ __forceinline__ int dev_bits(unsigned long long x) { return x ? 64 - __clzll((long long)x) : 0; }

// ---------------------------------------------------------------- cluster-wide
// A cluster of SQ_CS CTAs of SQ_T threads; each CTA holds up to sq_chunk<K>()
// sort items in shared memory, so one cluster sorts up to sq_max<K>() items
// (45,056 with 64-bit keys, 65,536 with 32-bit keys).
constexpr int SQ_CS = 8;                        // CTAs per cluster (portable size)
constexpr int SQ_T = 1024;                      // threads per CTA
// dynamic shared memory of a cluster-sort CTA: two key and two value buffers
// and the ranks of one pass, for sq_chunk<K>() items of key type K
constexpr size_t SQ_SMEM = 160 * 1024;
template <class K> __host__ __device__ constexpr int sq_chunk() {
    return (int)(SQ_SMEM / (2 * sizeof(K) + 3 * sizeof(uint32_t))) / 32 * 32;
}
template <class K> __host__ __device__ constexpr int sq_max() { return SQ_CS * sq_chunk<K>(); }
constexpr int SQ_RANK_MAX = 256;                // up to this many items one CTA ranks them directly

// the sort buffers of key type K in the dynamic shared memory
template <class K> struct SqBuf {
    K *ka, *kb;
    uint32_t *va, *vb, *rk;
    __device__ explicit SqBuf(unsigned char *smem) {
        ka = reinterpret_cast<K *>(smem);
        kb = ka + sq_chunk<K>();
        va = reinterpret_cast<uint32_t *>(kb + sq_chunk<K>());
        vb = va + sq_chunk<K>();
        rk = vb + sq_chunk<K>();
    }
};

// Stable LSD radix sort of the n pairs (keys[i], vals[i]) in global memory,
// in place, 8 bits per pass, by the whole cluster.  CTA r holds the items of
// global positions [r*chunk, (r+1)*chunk) in shared memory; per pass each CTA
// ranks its items by digit (stable: warp-major, slot-major, lane-minor, as
// the items lie in global order), publishes its per-digit counts, reads the
// other CTAs' counts, and writes each item into the shared-memory buffer of
// the CTA that holds its destination position.
template <class K>
__device__ __forceinline__ void cluster_radix_sort(cg::cluster_group &cl, K *keys, uint32_t *vals, int32_t n,
                                                   int passes, SqBuf<K> B, uint32_t *s_wc, uint32_t *s_tot,
                                                   uint32_t *s_base) {
    K *ka = B.ka, *kb = B.kb;
    uint32_t *va = B.va, *vb = B.vb, *rk = B.rk;
    if (n <= 1 || passes <= 0) return;   // uniform over the cluster
    const int r = (int)cl.block_rank(), t = threadIdx.x, T = blockDim.x, lane = t & 31, w = t >> 5;
    if (n <= SQ_RANK_MAX) {
        // few items: CTA 0 ranks them directly (stable: ties by position) on
        // the sorted bits, the other CTAs wait at the barrier
        if (r == 0) {
            const K mask = 8 * passes >= (int)(8 * sizeof(K)) ? ~K(0) : ((K(1) << (8 * passes)) - 1);
            for (int32_t i = t; i < n; i += T) {
                ka[i] = keys[i];
                va[i] = vals[i];
            }
            __syncthreads();
            for (int32_t i = t; i < n; i += T) {
                const K ki = ka[i] & mask;
                int32_t rank = 0;
                for (int32_t j = 0; j < n; j++) {
                    const K kj = ka[j] & mask;
                    rank += (kj < ki || (kj == ki && j < i)) ? 1 : 0;
                }
                keys[rank] = ka[i];
                vals[rank] = va[i];
            }
        }
        cl.sync();
        return;
    }
    const int nwarp = T >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const int32_t chunk = (n + SQ_CS - 1) / SQ_CS;
    const int32_t lo = min(n, r * chunk), hi = min(n, lo + chunk), mine_n = hi - lo;
    const int S = (chunk + T - 1) / T;
    for (int32_t i = t; i < mine_n; i += T) {
        ka[i] = keys[lo + i];
        va[i] = vals[lo + i];
    }
    for (int p = 0; p < passes; p++) {
        const int shift = 8 * p;
        uint32_t *run = s_wc + w * 256;
        for (int d = lane; d < 256; d += 32) run[d] = 0;
        __syncthreads();   // ka filled (first pass: the loads above; later passes: the cluster barrier)
        // rk[i] = (rank of item i among the warp's items of its digit) << 9 | digit
        for (int k = 0; k < S; k++) {
            const int32_t i = w * 32 * S + 32 * k + lane;
            const uint32_t d = i < mine_n ? ((uint32_t)(ka[i] >> shift) & 255u) : 256u;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            uint32_t base = 0;
            if (d < 256u) base = run[d];
            __syncwarp();
            if (i < mine_n) rk[i] = ((base + __popc(peers & lt)) << 9) | d;
            if (d < 256u && (peers & lt) == 0) run[d] = base + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // per digit: the warps' exclusive offsets inside this CTA, and the CTA total
        if (t < 256) {
            uint32_t acc = 0;
            for (int ww = 0; ww < nwarp; ww++) {
                const uint32_t x = s_wc[ww * 256 + t];
                s_wc[ww * 256 + t] = acc;
                acc += x;
            }
            s_tot[t] = acc;
        }
        cl.sync();   // every CTA's totals are published
        if (t < 256) {
            uint32_t below = 0, all = 0;
            for (int q = 0; q < SQ_CS; q++) {
                const uint32_t x = cl.map_shared_rank(s_tot, q)[t];
                all += x;
                if (q < r) below += x;
            }
            s_base[t] = below;
            s_base[256 + t] = all;
        }
        __syncthreads();
        // exclusive scan of the digit totals (one warp, 8 digits a lane)
        if (w == 0) {
            uint32_t v8[8], sum = 0;
#pragma unroll
            for (int k = 0; k < 8; k++) {
                v8[k] = s_base[256 + lane * 8 + k];
                sum += v8[k];
            }
            uint32_t inc = sum;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += u;
            }
            uint32_t run0 = inc - sum;
#pragma unroll
            for (int k = 0; k < 8; k++) {
                s_base[lane * 8 + k] += run0;   // digit start + earlier CTAs' items of the digit
                run0 += v8[k];
            }
        }
        __syncthreads();
        for (int k = 0; k < S; k++) {
            const int32_t i = w * 32 * S + 32 * k + lane;
            if (i < mine_n) {
                const uint32_t d = rk[i] & 511u;
                const uint32_t pos = s_base[d] + s_wc[w * 256 + d] + (rk[i] >> 9);
                const int q = (int)(pos / (uint32_t)chunk);
                const uint32_t at = pos - (uint32_t)q * (uint32_t)chunk;
                cl.map_shared_rank(kb, q)[at] = ka[i];
                cl.map_shared_rank(vb, q)[at] = va[i];
            }
        }
        cl.sync();   // every item has arrived in its new CTA
        K *tk = ka;
        ka = kb;
        kb = tk;
        uint32_t *tv = va;
        va = vb;
        vb = tv;
    }
    for (int32_t i = t; i < mine_n; i += T) {
        keys[lo + i] = ka[i];
        vals[lo + i] = va[i];
    }
    cl.sync();   // the sorted arrays are complete before anyone reads them
}

// exclusive prefix sum of in[0..n) into out, by one CTA, any integer type;
// in == out allowed
template <class T>
__device__ __forceinline__ void block_scan_excl_t(const T *in, T *out, int64_t n, T *s_tmp) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T carry = 0;
    for (int64_t base = 0; base < n; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const T x = i < n ? in[i] : T(0);
        T inc = x;
        for (int o = 1; o < 32; o <<= 1) {
            const T u = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += u;
        }
        if (lane == 31) s_tmp[wid] = inc;
        __syncthreads();
        if (wid == 0) {
            const T y = lane < nw ? s_tmp[lane] : T(0);
            T yi = y;
            for (int o = 1; o < 32; o <<= 1) {
                const T u = __shfl_up_sync(0xffffffffu, yi, o);
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

// exclusive prefix sum of in[0..n) into out by the cluster (in == out
// allowed); returns the total.  s_tmp: 33 words, s_part: 1 word of shared
// memory.
template <class T>
__device__ __forceinline__ T cluster_scan_excl(cg::cluster_group &cl, const T *in, T *out, int32_t n, T *s_tmp,
                                               T *s_part) {
    const int r = (int)cl.block_rank(), t = threadIdx.x;
    const int32_t chunk = (n + SQ_CS - 1) / SQ_CS;
    const int32_t lo = min(n, r * chunk), hi = min(n, lo + chunk);
    // the CTA's own total first (in may be overwritten by the local scan)
    T loc = 0;
    for (int32_t i = lo + t; i < hi; i += blockDim.x) loc += in[i];
    for (int o = 16; o > 0; o >>= 1) loc += __shfl_down_sync(0xffffffffu, loc, o);
    if ((t & 31) == 0) s_tmp[t >> 5] = loc;
    __syncthreads();
    if (t == 0) {
        T sum = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) sum += s_tmp[k];
        *s_part = sum;
    }
    __syncthreads();
    block_scan_excl_t<T>(in + lo, out + lo, hi - lo, s_tmp);
    cl.sync();
    T off = 0, total = 0;
    for (int q = 0; q < SQ_CS; q++) {
        const T x = *cl.map_shared_rank(s_part, q);
        if (q < r) off += x;
        total += x;
    }
    if (off)
        for (int32_t i = lo + t; i < hi; i += blockDim.x) out[i] += off;
    cl.sync();
    return total;
}

// sum of x over the cluster (every thread of every CTA takes part)
__device__ __forceinline__ int32_t cluster_sum_i32(cg::cluster_group &cl, int32_t x, int32_t *s_tmp, int32_t *s_part) {
    x = block_sum(x, s_tmp);
    if (threadIdx.x == 0) *s_part = x;
    cl.sync();
    int32_t total = 0;
    for (int q = 0; q < SQ_CS; q++) total += *cl.map_shared_rank(s_part, q);
    cl.sync();
    return total;
}

// maximum over the cluster (every thread of every CTA takes part)
__device__ __forceinline__ long long cluster_max_ll(cg::cluster_group &cl, long long x, long long *s_ll) {
    x = block_max_ll(x, s_ll);
    if (threadIdx.x == 0) s_ll[33] = x;
    cl.sync();
    long long m = LLONG_MIN;
    for (int q = 0; q < SQ_CS; q++) m = max(m, cl.map_shared_rank(s_ll, q)[33]);
    cl.sync();   // nobody overwrites s_ll[33] before every CTA has read it
    return m;
}

// the maxima of three values over the cluster, in place (every thread of
// every CTA takes part; s_ll holds 40 words)
__device__ __forceinline__ void cluster_max3_ll(cg::cluster_group &cl, long long &a, long long &b, long long &c,
                                                long long *s_ll) {
    a = block_max_ll(a, s_ll);
    b = block_max_ll(b, s_ll);
    c = block_max_ll(c, s_ll);
    if (threadIdx.x == 0) {
        s_ll[34] = a;
        s_ll[35] = b;
        s_ll[36] = c;
    }
    cl.sync();
    for (int q = 0; q < SQ_CS; q++) {
        const long long *o = cl.map_shared_rank(s_ll, q);
        a = max(a, o[34]);
        b = max(b, o[35]);
        c = max(c, o[36]);
    }
    cl.sync();   // nobody overwrites s_ll[34..36] before every CTA has read them
}

}  // namespace hp
