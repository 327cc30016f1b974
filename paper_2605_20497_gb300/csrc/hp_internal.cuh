// hp_internal.cuh -- shared declarations of the CUDA partitioner (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <stdexcept>
#include <string>
#include <utility>
#include <vector>

#include "hp.h"

namespace hp {

// ---------------------------------------------------------------- errors
struct Error : std::runtime_error {
    hp_status status;
    Error(hp_status s, const std::string &m) : std::runtime_error(m), status(s) {}
};

void cuda_check(cudaError_t e, const char *what, const char *file, int line);
#define HPC(x) ::hp::cuda_check((x), #x, __FILE__, __LINE__)
// every kernel launch is followed by this check, which also counts the launch
extern thread_local int64_t t_launches;
#define HP_LAUNCH_CHECK() \
    (::hp::t_launches++, ::hp::cuda_check(cudaGetLastError(), "kernel launch", __FILE__, __LINE__))

// ---------------------------------------------------------------- launches
// Every kernel of the path is launched with programmatic stream
// serialisation: a kernel may be scheduled while the one before it on the
// stream is still running, so that its launch and block set-up overlap the
// predecessor's tail (the path is a chain of tens of thousands of short
// dependent kernels).  Each kernel therefore starts with HP_KERNEL_ENTER():
// its threads wait there until the preceding kernel has finished and its
// writes are visible (before any read or write of memory), then allow the
// next kernel to be scheduled.  Work issued to a stream other than as a
// kernel (copies, memsets, event waits) keeps the full ordering.
#define HP_KERNEL_ENTER()                                          \
    do {                                                           \
        asm volatile("griddepcontrol.wait;" ::: "memory");         \
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); \
    } while (0)

// launches are made with the attribute unless HP_PDL=0 was set in the
// environment when the library first launched a kernel, or the calling
// thread set t_plain_launches.  The batch workers set it: with many streams
// in flight, a kernel's blocks waiting at entry for their predecessor hold
// SM slots that the other streams' kernels would use.
extern thread_local bool t_plain_launches;
bool pdl_enabled();

// Plain launches while in scope if `on` (nested scopes keep an outer
// setting).  The level loop uses it for levels of more than PDL_MAX_N nodes:
// their kernels are long and several run side by side on side streams, where
// blocks waiting at entry only take SM slots from the other stream (measured:
// 1M-node Gaussian net 1.68 s plain, 1.79 s with the attribute everywhere);
// the chains of short kernels of the smaller levels gain from it.
constexpr int32_t PDL_MAX_N = 32768;
struct PlainLaunchScope {
    bool prev;
    explicit PlainLaunchScope(bool on) : prev(t_plain_launches) { t_plain_launches = prev || on; }
    ~PlainLaunchScope() { t_plain_launches = prev; }
};

template <class... E, class... A>
inline void launch_k(void (*kernel)(E...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A &&...args) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    cuda_check(cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...), "kernel launch", __FILE__, __LINE__);
}

// bits of the device error word
enum : uint32_t {
    E_OFFSETS = 1u,
    E_PIN = 2u,
    E_SRC = 4u,
    E_DUP = 8u,
    E_WEIGHT = 16u,
    E_WSUM = 32u,
    E_INFEAS = 64u,
    E_TIMEOUT = 128u,
    E_INTERNAL = 256u,
};

// ---------------------------------------------------------------- memory
// Stream-ordered device workspace; everything still held is released by the
// destructor (on the same stream).
class Arena {
  public:
    explicit Arena(cudaStream_t s) : stream_(s) {}
    ~Arena();
    Arena(const Arena &) = delete;
    Arena &operator=(const Arena &) = delete;
    void *raw(size_t bytes);
    template <class T> T *get(size_t n) { return static_cast<T *>(raw(n * sizeof(T))); }
    void release(void *p);
    cudaStream_t stream() const { return stream_; }

  private:
    cudaStream_t stream_;
    std::vector<void *> live_;
};

// small pinned host mailbox for device -> host reads of counters
template <class T> T fetch(const T *dptr, cudaStream_t s);
void fetch_bytes(void *host, const void *dev, size_t bytes, cudaStream_t s);

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int bits_for(uint64_t maxval) {
    int b = 0;
    while (b < 64 && (maxval >> b) != 0) b++;
    return b;
}
int num_sms();

// ---------------------------------------------------------------- primitives
// exclusive prefix sum of n elements; *total_dev (device, optional) = sum.
void scan_excl(const int32_t *in, int32_t *out, int64_t n, int32_t *total_dev, Arena &A);
void scan_excl(const int64_t *in, int64_t *out, int64_t n, int64_t *total_dev, Arena &A);
// stable LSD radix sort of (key, value) pairs on the low `bits` bits of key.
void radix_sort(uint32_t *keys, uint32_t *vals, int64_t n, int bits, Arena &A);
void radix_sort(uint64_t *keys, uint32_t *vals, int64_t n, int bits, Arena &A);
// the same with the element count in device memory (*n_dev <= cap); stable
void radix_sort_dev(uint32_t *keys, uint32_t *vals, const int32_t *n_dev, int64_t cap, int bits, Arena &A);
void radix_sort_dev(uint64_t *keys, uint32_t *vals, const int32_t *n_dev, int64_t cap, int bits, Arena &A);
void fill_i32(int32_t *p, int64_t n, int32_t v, cudaStream_t s);
void iota_i32(int32_t *p, int64_t n, cudaStream_t s);

// Stable LSD radix sort of (keys[i], vals[i]), i < n <= cap, by one CTA of
// any multiple of 32 threads (up to 1024), on the low 8*passes bits.
// smem: 2*cap*(sizeof(K)+4) bytes; s_wc: 32*256 words; s_hist: 256 words.
// Per pass: digit histogram, its exclusive scan, then rounds of blockDim
// items in index order ranked within a warp by match and across warps by
// per-warp digit counts.  Ends with the sorted data back in keys/vals and a
// __syncthreads.
// Stable LSD radix sort (8-bit digits) of n (key, value) pairs by one CTA of
// up to 1024 threads, n <= 16 * blockDim.x.  keys/vals are staged in two
// pairs of buffers ka/kb, va/vb of >= n entries (shared or global memory);
// s_wc holds 32 * 256 counters, s_hist 256 + 33 words.  Warp w owns items [w * 32S, (w + 1) * 32S)
// with S = ceil(n / blockDim.x), slot k of lane l being item w * 32S + 32k + l,
// so one round per pass ranks every item: within a warp slot by slot
// (match_any), then across warps by an exclusive scan over (digit, warp).
constexpr int BRS_SLOTS = 16;
template <class K>
__device__ void block_radix_sort_buf(K *keys, uint32_t *vals, int n, int passes, K *ka, K *kb, uint32_t *va,
                                     uint32_t *vb, uint32_t *s_wc, uint32_t *s_hist) {
    const int t = threadIdx.x, T = blockDim.x, lane = t & 31, w = t >> 5, nwarp = T >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    __syncthreads();
    if (n <= 1) return;
    const int S = (n + T - 1) / T;
    for (int i = t; i < n; i += T) {
        ka[i] = keys[i];
        va[i] = vals[i];
    }
    __syncthreads();
    for (int p = 0; p < passes; p++) {
        const int shift = 8 * p;
        uint32_t *run = s_wc + w * 256;
        for (int d = lane; d < 256; d += 32) run[d] = 0;
        __syncwarp();
        uint32_t mine[BRS_SLOTS];   // rank << 9 | digit (256 = no item)
#pragma unroll
        for (int k = 0; k < BRS_SLOTS; k++) {
            if (k < S) {
                const int i = w * 32 * S + 32 * k + lane;
                const uint32_t d = i < n ? ((uint32_t)(ka[i] >> shift) & 255u) : 256u;
                const uint32_t peers = __match_any_sync(0xffffffffu, d);
                uint32_t base = 0;
                if (d < 256u) base = run[d];
                __syncwarp();
                mine[k] = ((base + __popc(peers & lt)) << 9) | d;
                if (d < 256u && (peers & lt) == 0) run[d] = base + __popc(peers);
                __syncwarp();
            }
        }
        __syncthreads();
        // exclusive scan over the (digit, warp) counters, digit-major: thread
        // t takes the counters of digits [8t / nwarp ...) in groups of 8
        const int total = 256 * nwarp;
        const int per = (total + T - 1) / T;
        uint32_t loc = 0;
        for (int q = 0; q < per; q++) {
            const int e = t * per + q;
            if (e < total) loc += s_wc[(e % nwarp) * 256 + e / nwarp];
        }
        uint32_t inc = loc;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += u;
        }
        if (lane == 31) s_hist[w] = inc;
        __syncthreads();
        if (w == 0) {
            const uint32_t y = lane < nwarp ? s_hist[lane] : 0u;
            uint32_t yi = y;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, yi, o);
                if (lane >= o) yi += u;
            }
            if (lane < nwarp) s_hist[256 + lane] = yi - y;
        }
        __syncthreads();
        uint32_t off = s_hist[256 + w] + inc - loc;
        for (int q = 0; q < per; q++) {
            const int e = t * per + q;
            if (e < total) {
                uint32_t *c = &s_wc[(e % nwarp) * 256 + e / nwarp];
                const uint32_t x = *c;
                *c = off;
                off += x;
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < BRS_SLOTS; k++) {
            if (k < S && (mine[k] & 511u) < 256u) {
                const int i = w * 32 * S + 32 * k + lane;
                const uint32_t pos = s_wc[w * 256 + (mine[k] & 511u)] + (mine[k] >> 9);
                kb[pos] = ka[i];
                vb[pos] = va[i];
            }
        }
        __syncthreads();
        K *tk = ka;
        ka = kb;
        kb = tk;
        uint32_t *tv = va;
        va = vb;
        vb = tv;
    }
    for (int i = t; i < n; i += T) {
        keys[i] = ka[i];
        vals[i] = va[i];
    }
    __syncthreads();
}

// the same with both buffer pairs carved out of `smem` (`cap` entries each)
template <class K>
__device__ void block_radix_sort(K *keys, uint32_t *vals, int n, int passes, int cap, unsigned char *smem,
                                 uint32_t *s_wc, uint32_t *s_hist) {
    K *ka = reinterpret_cast<K *>(smem);
    K *kb = ka + cap;
    uint32_t *va = reinterpret_cast<uint32_t *>(kb + cap);
    uint32_t *vb = va + cap;
    block_radix_sort_buf<K>(keys, vals, n, passes, ka, kb, va, vb, s_wc, s_hist);
}

// Segmented sum over runs of equal, non-decreasing keys within a warp: every
// lane passes its key and value; returns true on the last lane of its run
// (whose *acc then holds the run's total within the warp).  All 32 lanes
// must take part.
template <class T> __device__ __forceinline__ bool warp_run_sum(int32_t key, T &acc) {
    const int lane = threadIdx.x & 31;
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, acc, o);
        int32_t k = __shfl_up_sync(0xffffffffu, key, o);
        if (lane >= o && k == key) acc += y;
    }
    int32_t nk = __shfl_down_sync(0xffffffffu, key, 1);
    return lane == 31 || nk != key;
}

// Per-thread write combining for hub nodes: a few (key, sum, count) entries
// in registers absorb repeated updates of the same key; an evicted or final
// entry is flushed by the caller-supplied functor (one atomic per flush).
// Sums are integers, so the result does not depend on the flush order.
template <int K> struct RegCache {
    int32_t key[K];
    unsigned long long sum[K];
    uint32_t cnt[K];
    int next;
    __device__ void init() {
#pragma unroll
        for (int i = 0; i < K; i++) key[i] = -1;
        next = 0;
    }
    template <class F> __device__ void add(int32_t k, unsigned long long v, uint32_t c, F &&flush) {
#pragma unroll
        for (int i = 0; i < K; i++)
            if (key[i] == k) {
                sum[i] += v;
                cnt[i] += c;
                return;
            }
        int slot = next;
        next = (next + 1) % K;
#pragma unroll
        for (int i = 0; i < K; i++)
            if (i == slot) {
                if (key[i] >= 0) flush(key[i], sum[i], cnt[i]);
                key[i] = k;
                sum[i] = v;
                cnt[i] = c;
            }
    }
    template <class F> __device__ void drain(F &&flush) {
#pragma unroll
        for (int i = 0; i < K; i++)
            if (key[i] >= 0) {
                flush(key[i], sum[i], cnt[i]);
                key[i] = -1;
            }
    }
};

// kernel attributes: raises the dynamic shared memory limit of `func` to
// `smem` once and returns its resident CTAs per SM (cached per pair)
int prepare_kernel(const void *func, int block, size_t smem);

// ---------------------------------------------------------------- levels
// One hypergraph of the hierarchy, device resident.
struct Level {
    int32_t n = 0, e = 0;
    int64_t np = 0;
    int32_t *off = nullptr;    // [e+1] hyperedge segments: src pins first, then dst pins
    int32_t *pin = nullptr;    // [np]
    int32_t *pedge = nullptr;  // [np] hyperedge of every pin position
    int32_t *nsrc = nullptr;   // [e] |src(e)|
    int32_t *size = nullptr;   // [n] node sizes
    int32_t *ioff = nullptr;   // [n+1] incidence segments
    int32_t *inc = nullptr;    // [np] in(v) ascending, then out(v) ascending
    int32_t *inode = nullptr;  // [np] node of every incidence entry
    int32_t *nin = nullptr;    // [n] |in(v)|
    int32_t *gamma = nullptr;  // [n] node -> node of the next level
    int32_t *nbnd = nullptr;   // [n] upper bound on |N(v)| (neighbour table sizing)
};

struct Params {
    int32_t omega, delta;
    uint64_t seed;
    hp_options o;
    int64_t wsum = 0;   // sum of hyperedge weights (bounds any gain)
};

// graph construction (hp_graph.cu)
uint32_t validate_and_build_level0(const int32_t *pins, const int32_t *offsets, int32_t e, int32_t n,
                                   const int32_t *src_counts, const int32_t *weights, Params &P, Level &L,
                                   int32_t *w_out, Arena &A);
void build_incidence(Level &L, Arena &A);
// level graph from caller arrays (device): copies them and builds the incidence
void make_level(int32_t n, int32_t e, const int32_t *off, const int32_t *pins, const int32_t *nsrc,
                const int32_t *size, Level &L, Arena &A);
// device counters of one coarsening level (read by the host once per level)
struct LevelBox {
    unsigned long long qsum, visits, pairs, iso, nbrs;
    uint64_t cap;      // noise cap of the level
    int32_t cn, cnp;   // nodes and pins of the coarse level
    uint32_t err;      // error bits raised by the level's matching
    int32_t isolist;   // nodes without a valid neighbour (the best-effort pairing's list)
    int32_t ntargets;  // distinct targets of the first proposal graph
    int32_t maxin;     // largest in-degree of the first proposal graph
    unsigned long long pairs1;   // pairs of the first matching round
};
// Contraction (Sec. V-E): computes the coarse sizes into box_dev, reads the
// box once into box_host; returns false and builds nothing when the level
// formed no pair.
bool contract_level(const Level &L, const int32_t *mate, LevelBox *box_dev, LevelBox *box_host, Level &C, Arena &A);

// loads the no-allocation entry point's module on the current device, once
// per device (hp_noalloc.cu)
void noalloc_prepare();

// coarsening (hp_coarsen.cu)
struct CoarsenWs;
CoarsenWs *coarsen_workspace(int32_t n, int32_t e, const Params &P, Arena &A);
void coarsen_workspace_free(CoarsenWs *W, Arena &A);
LevelBox *coarsen_box(CoarsenWs *W);
// One level on the device, no host synchronisation; counters in the box.
// prop_events (optional): two events recorded around the proposal launches
void coarsen_level(Level &L, int32_t level, const int32_t *w, const Params &P, int32_t *mate, CoarsenWs &W, Arena &A,
                   uint32_t *err_dev, int32_t *cand_out = nullptr, uint64_t *score_out = nullptr,
                   cudaEvent_t *prop_events = nullptr);

// learned merge priority (hp_learned.cu)
bool merge_model_ok(const hp_merge_model &m);
struct LearnIn {
    int32_t n, K, pi, level, omega, delta;
    // nodes [v0, v1) are scored by one pass; feat, rank and score hold the
    // rows of those nodes only, row (v - v0) * K + j (the whole level: 0, n)
    int32_t v0 = 0, v1 = 0;
    const int32_t *size, *ioff, *inc, *nin;   // the level graph
    const int32_t *candK;                     // [n*K] top-K valid neighbours by (eta, id), -1 padded
    const uint64_t *csK;                      // [n*K] their eta (with noise)
    const hp_merge_model *model;              // device copy
    uint8_t *feat;                            // [(v1-v0)*K][16] scratch, 16-byte aligned
    int32_t *rank;                            // [(v1-v0)*K] scratch
    int32_t *score;                           // [(v1-v0)*K] scratch
    int32_t *cand;                            // [n*pi] out: C(n)
    uint64_t *cscore;                         // [n*pi] out: eta of C(n)
};
// C(n) of every node, in passes of `batch` nodes (0: one pass); X.feat,
// X.rank and X.score hold batch * K rows
void learned_candidates(LearnIn X, int32_t batch, cudaStream_t s);
void merge_features(const LearnIn &X, cudaStream_t s);   // k_merge_feats alone into X.feat / X.rank
// level-0 top-K lists (K = P.o.learned_k) and the features of every listed pair
void level_features(Level &L, const int32_t *w, const Params &P, CoarsenWs &W, Arena &A, uint32_t *err_dev,
                    int32_t *cand_out, int32_t *rank_out, uint8_t *feat_out);
// training of the merge MLP: mean loss and gradient (synchronises), AdamW step, integer model
double merge_grad(const uint8_t *feat, const float *label, int64_t count, const float *params, float *grad,
                  Arena &A);
void merge_adam(float *p, const float *g, float *m, float *v, int64_t step, float lr, float b1, float b2, float eps,
                float wd, cudaStream_t s);
void merge_quantize(const float *params, const uint8_t *calib, int64_t count, hp_merge_model &M);
void merge_scores(const uint8_t *feat, int64_t count, const hp_merge_model *dmodel, int32_t *out, cudaStream_t s);

// refinement (hp_refine.cu)
// optional copies of the intermediate results of one repetition (device
// buffers of n entries; m and best_gain are host / device scalars)
struct RepDebug {
    int32_t *node, *src, *dst;   // proposed moves, sorted (p_s asc, gain desc, node asc)
    long long *gain;
    int32_t *seq;                // seq[k] = index (into the sorted moves) of the k-th move of the sequence
    long long *gseq;             // in-sequence gain of the k-th move
    long long *best_gain;        // device scalar
    int32_t *m;                  // host: number of moves
};
int32_t refine_rep_debug(const Level &L, const int32_t *w, int32_t nparts, const Params &P, int32_t *rho,
                         int second_half, Arena &A, uint32_t *err_dev, const RepDebug &dbg);
struct RefineOut {
    int64_t moves = 0;
    int32_t reps = 0;
    int64_t alg_bytes = 0;   // algorithmic bytes of the level's repetitions
};
struct LevelWs;
// refinement workspace for levels of at most n nodes, np pins, e hyperedges
// and max_e pins per hyperedge (the level-0 sizes)
LevelWs *refine_workspace(int32_t n, int64_t np, int32_t e, int32_t nparts, int32_t max_e, const Params &P,
                          Arena &A);
void refine_workspace_free(LevelWs *W, Arena &A);
int32_t max_edge_size(const Level &L, Arena &A);
RefineOut refine_level(const Level &L, const int32_t *w, const Params &P, int32_t *rho, LevelWs *W, Arena &A,
                       uint32_t *err_dev);
void objective(const Level &L, const int32_t *w, const int32_t *rho, int32_t nparts, int64_t *conn_dev,
               int64_t *cutnet_dev, Arena &A);
void part_stats(const Level &L, const int32_t *w, const int32_t *part, int32_t nparts, int32_t omega, int32_t delta,
                int64_t *out, Arena &A);

// allocator hook (hp_prims.cu)
void set_allocator(void *(*a)(size_t, void *), void (*f)(void *, void *), void *ctx);

}  // namespace hp
