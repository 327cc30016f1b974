// hp_prims.cu -- workspace, device->host mailbox, prefix sums and a stable
// LSD radix sort (the sort/scan patterns of Sec. VI-C and VI-D, also used to
// build incidence sets).
#include <cuda_runtime.h>

#include <cstdlib>

#include <cstring>
#include <mutex>

#include "hp_internal.cuh"

namespace hp {

thread_local int64_t t_launches = 0;

// ================================================================ errors
void cuda_check(cudaError_t e, const char *what, const char *file, int line) {
    if (e == cudaSuccess) return;
    std::string m = std::string(what) + ": " + cudaGetErrorString(e) + " (" + file + ":" + std::to_string(line) + ")";
    if (e == cudaErrorMemoryAllocation) throw Error(HP_ERR_OOM, m);
    throw Error(HP_ERR_CUDA, m);
}

// ================================================================ memory
static void *(*g_alloc)(size_t, void *) = nullptr;
static void (*g_free)(void *, void *) = nullptr;
static void *g_ctx = nullptr;

void set_allocator(void *(*a)(size_t, void *), void (*f)(void *, void *), void *ctx) {
    g_alloc = a;
    g_free = f;
    g_ctx = ctx;
}

static cudaMemPool_t device_pool() {
    static std::mutex mu;
    static std::vector<cudaMemPool_t> pools;
    int dev = 0;
    HPC(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if ((int)pools.size() <= dev) pools.resize(dev + 1, nullptr);
    if (!pools[dev]) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof props);
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        HPC(cudaMemPoolCreate(&pools[dev], &props));
        uint64_t keep = ~0ull;  // keep freed blocks for reuse by later calls
        HPC(cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep));
    }
    return pools[dev];
}

void *Arena::raw(size_t bytes) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    void *p = nullptr;
    if (g_alloc) {
        p = g_alloc(bytes, g_ctx);
        if (!p) throw Error(HP_ERR_OOM, "workspace allocation of " + std::to_string(bytes) + " bytes failed");
    } else {
        cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, device_pool(), stream_);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            throw Error(HP_ERR_OOM, "workspace allocation of " + std::to_string(bytes) + " bytes failed");
        }
    }
    live_.push_back(p);
    return p;
}

void Arena::release(void *p) {
    if (!p) return;
    for (size_t i = 0; i < live_.size(); i++)
        if (live_[i] == p) {
            if (g_free) g_free(p, g_ctx);
            else (void)cudaFreeAsync(p, stream_);
            live_[i] = live_.back();
            live_.pop_back();
            return;
        }
}

Arena::~Arena() {
    for (void *p : live_) {
        if (g_free) g_free(p, g_ctx);
        else (void)cudaFreeAsync(p, stream_);
    }
    (void)cudaStreamSynchronize(stream_);
}

static thread_local void *t_mailbox = nullptr;
static const size_t kMailbox = 1 << 16;

void fetch_bytes(void *host, const void *dev, size_t bytes, cudaStream_t s) {
    if (bytes > kMailbox) {
        HPC(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, s));
        HPC(cudaStreamSynchronize(s));
        return;
    }
    if (!t_mailbox) HPC(cudaMallocHost(&t_mailbox, kMailbox));
    HPC(cudaMemcpyAsync(t_mailbox, dev, bytes, cudaMemcpyDeviceToHost, s));
    HPC(cudaStreamSynchronize(s));
    std::memcpy(host, t_mailbox, bytes);
}

template <class T> T fetch(const T *dptr, cudaStream_t s) {
    T v;
    fetch_bytes(&v, dptr, sizeof(T), s);
    return v;
}
template int32_t fetch<int32_t>(const int32_t *, cudaStream_t);
template int64_t fetch<int64_t>(const int64_t *, cudaStream_t);
template uint32_t fetch<uint32_t>(const uint32_t *, cudaStream_t);
template uint64_t fetch<uint64_t>(const uint64_t *, cudaStream_t);
template unsigned long long fetch<unsigned long long>(const unsigned long long *, cudaStream_t);
template long long fetch<long long>(const long long *, cudaStream_t);
template double fetch<double>(const double *, cudaStream_t);

int prepare_kernel(const void *func, int block, size_t smem) {
    // per (kernel, device): the dynamic shared memory limit is set on first
    // use and only ever grows, so a size admitted once stays admitted;
    // occupancy cached per size
    struct Entry {
        const void *f;
        int dev, block;
        size_t smem;
        int occ;
    };
    static std::mutex mu;
    static std::vector<Entry> occ_cache;
    static std::vector<std::pair<std::pair<const void *, int>, size_t>> limit;
    int dev = 0;
    HPC(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    size_t *lim = nullptr;
    for (auto &l : limit)
        if (l.first.first == func && l.first.second == dev) lim = &l.second;
    if (!lim) {
        // nothing assumed: without the attribute a kernel gets 48 KB minus
        // its static shared memory, so the first request always sets it
        limit.push_back({{func, dev}, (size_t)0});
        lim = &limit.back().second;
    }
    if (smem > *lim) {
        HPC(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        *lim = smem;
    }
    for (auto &c : occ_cache)
        if (c.f == func && c.dev == dev && c.block == block && c.smem == smem) return c.occ;
    int occ = 0;
    HPC(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, func, block, smem));
    occ = std::max(occ, 1);
    occ_cache.push_back({func, dev, block, smem, occ});
    return occ;
}

thread_local bool t_plain_launches = false;

bool pdl_enabled() {
    static const bool on = [] {
        const char *e = std::getenv("HP_PDL");
        return !(e && e[0] == '0');
    }();
    return on && !t_plain_launches;
}

int num_sms() {
    static int sms[64] = {0};
    int dev = 0;
    HPC(cudaGetDevice(&dev));
    if (dev < 64 && sms[dev]) return sms[dev];
    int v = 0;
    HPC(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
    if (dev < 64) sms[dev] = v;
    return v;
}

// ================================================================ fill / iota
__global__ void k_fill(int32_t *p, int64_t n, int32_t v) {
    HP_KERNEL_ENTER();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}
__global__ void k_iota(int32_t *p, int64_t n) {
    HP_KERNEL_ENTER();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (int32_t)i;
}
static int grid_for(int64_t n, int block) {
    int64_t g = cdiv(n, block);
    int64_t cap = (int64_t)num_sms() * 16;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}
void fill_i32(int32_t *p, int64_t n, int32_t v, cudaStream_t s) {
    if (n <= 0) return;
    launch_k(k_fill, grid_for(n, 256), 256, 0, s, p, n, v);
    HP_LAUNCH_CHECK();
}
void iota_i32(int32_t *p, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    launch_k(k_iota, grid_for(n, 256), 256, 0, s, p, n);
    HP_LAUNCH_CHECK();
}

// ================================================================ scan
// Tile of 512 threads x 8 items: per-tile sums, scan of the sums (recursive),
// then per-tile exclusive scans with the tile offset.
constexpr int SCAN_T = 512, SCAN_I = 8, SCAN_TILE = SCAN_T * SCAN_I;

template <class T> __device__ T warp_incl_scan(T v) {
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) >= o) v += u;
    }
    return v;
}

template <class T> __device__ T block_excl_scan(T v, T *s_warp, T *total) {
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T inc = warp_incl_scan(v);
    if (lane == 31) s_warp[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        T x = lane < nw ? s_warp[lane] : T(0);
        T xi = warp_incl_scan(x);
        if (lane < nw) s_warp[lane] = xi - x;
        if (lane == nw - 1) s_warp[32] = xi;
    }
    __syncthreads();
    T r = inc - v + s_warp[wid];
    if (total) *total = s_warp[32];
    __syncthreads();
    return r;
}

template <class T> __global__ void __launch_bounds__(SCAN_T) k_scan_reduce(const T *in, T *bsum, int64_t n) {
    HP_KERNEL_ENTER();
    __shared__ T s_warp[33];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    T acc = 0;
    for (int i = 0; i < SCAN_I; i++) {
        int64_t k = base + (int64_t)i * SCAN_T + threadIdx.x;
        if (k < n) acc += in[k];
    }
    T tot;
    (void)block_excl_scan(acc, s_warp, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

template <class T>
__global__ void __launch_bounds__(SCAN_T) k_scan_tiles(const T *in, T *out, const T *boff, int64_t n, T *total) {
    HP_KERNEL_ENTER();
    __shared__ T s_val[SCAN_TILE];
    __shared__ T s_warp[33];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    for (int i = 0; i < SCAN_I; i++) {
        int64_t k = base + (int64_t)i * SCAN_T + threadIdx.x;
        s_val[i * SCAN_T + threadIdx.x] = k < n ? in[k] : T(0);
    }
    __syncthreads();
    T loc[SCAN_I];
    T acc = 0;
    for (int i = 0; i < SCAN_I; i++) {
        loc[i] = s_val[threadIdx.x * SCAN_I + i];
        acc += loc[i];
    }
    T tile_tot;
    T pre = block_excl_scan(acc, s_warp, &tile_tot);
    T off = boff ? boff[blockIdx.x] : T(0);
    T run = pre + off;
    for (int i = 0; i < SCAN_I; i++) {
        s_val[threadIdx.x * SCAN_I + i] = run;
        run += loc[i];
    }
    __syncthreads();
    for (int i = 0; i < SCAN_I; i++) {
        int64_t k = base + (int64_t)i * SCAN_T + threadIdx.x;
        if (k < n) out[k] = s_val[i * SCAN_T + threadIdx.x];
    }
    if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total = off + tile_tot;
}

// up to SCAN_SINGLE tiles: one CTA walks the tiles with a running carry
// (one launch instead of three)
constexpr int64_t SCAN_SINGLE = 4;
template <class T> __global__ void __launch_bounds__(SCAN_T) k_scan_single(const T *in, T *out, int64_t n, T *total) {
    HP_KERNEL_ENTER();
    __shared__ T s_val[SCAN_TILE];
    __shared__ T s_warp[33];
    T carry = 0;
    for (int64_t base = 0; base < n; base += SCAN_TILE) {
        for (int i = 0; i < SCAN_I; i++) {
            const int64_t k = base + (int64_t)i * SCAN_T + threadIdx.x;
            s_val[i * SCAN_T + threadIdx.x] = k < n ? in[k] : T(0);
        }
        __syncthreads();
        T loc[SCAN_I];
        T acc = 0;
        for (int i = 0; i < SCAN_I; i++) {
            loc[i] = s_val[threadIdx.x * SCAN_I + i];
            acc += loc[i];
        }
        T tile_tot;
        T run = block_excl_scan(acc, s_warp, &tile_tot) + carry;
        for (int i = 0; i < SCAN_I; i++) {
            s_val[threadIdx.x * SCAN_I + i] = run;
            run += loc[i];
        }
        __syncthreads();
        for (int i = 0; i < SCAN_I; i++) {
            const int64_t k = base + (int64_t)i * SCAN_T + threadIdx.x;
            if (k < n) out[k] = s_val[i * SCAN_T + threadIdx.x];
        }
        carry += tile_tot;
        __syncthreads();
    }
    if (total && threadIdx.x == 0) *total = carry;
}

template <class T> static void scan_impl(const T *in, T *out, int64_t n, T *total_dev, Arena &A) {
    cudaStream_t s = A.stream();
    if (n <= 0) {
        if (total_dev) HPC(cudaMemsetAsync(total_dev, 0, sizeof(T), s));
        return;
    }
    int64_t tiles = cdiv(n, SCAN_TILE);
    if (tiles <= SCAN_SINGLE) {
        launch_k(k_scan_single<T>, 1, SCAN_T, 0, s, in, out, n, total_dev);
        HP_LAUNCH_CHECK();
        return;
    }
    T *bsum = A.get<T>(tiles);
    T *boff = A.get<T>(tiles);
    launch_k(k_scan_reduce<T>, (unsigned)tiles, SCAN_T, 0, s, in, bsum, n);
    HP_LAUNCH_CHECK();
    scan_impl<T>(bsum, boff, tiles, nullptr, A);
    launch_k(k_scan_tiles<T>, (unsigned)tiles, SCAN_T, 0, s, in, out, boff, n, total_dev);
    HP_LAUNCH_CHECK();
    A.release(bsum);
    A.release(boff);
}

void scan_excl(const int32_t *in, int32_t *out, int64_t n, int32_t *total_dev, Arena &A) {
    scan_impl<int32_t>(in, out, n, total_dev, A);
}
void scan_excl(const int64_t *in, int64_t *out, int64_t n, int64_t *total_dev, Arena &A) {
    scan_impl<int64_t>(in, out, n, total_dev, A);
}

// ================================================================ radix sort
// 8-bit digits; a tile is 256 threads x 16 rounds.  Pass = per-tile digit
// histograms (digit-major), one exclusive scan, then a stable scatter where
// every round ranks its 256 items with warp match + per-warp counts.
constexpr int RS_T = 256, RS_R = 16, RS_TILE = RS_T * RS_R;

template <class K>
__global__ void __launch_bounds__(RS_T) k_radix_hist(const K *keys, int64_t n, int shift, uint32_t *hist, int tiles) {
    HP_KERNEL_ENTER();
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_R; r++) {
        int64_t i = base + (int64_t)r * RS_T + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(uint32_t)(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * tiles + blockIdx.x] = cnt[threadIdx.x];
}

template <class K>
__global__ void __launch_bounds__(RS_T) k_radix_scatter(const K *kin, const uint32_t *vin, K *kout, uint32_t *vout,
                                                        int64_t n, int shift, const uint32_t *offs, int tiles) {
    HP_KERNEL_ENTER();
    __shared__ uint32_t s_off[256];
    __shared__ uint32_t s_wc[8][256];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    s_off[t] = offs[(int64_t)t * tiles + blockIdx.x];
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_R; r++) {
        int64_t i0 = base + (int64_t)r * RS_T;
        if (i0 >= n) break;
        int64_t i = i0 + t;
        bool valid = i < n;
        K key = valid ? kin[i] : K(0);
        uint32_t val = valid ? vin[i] : 0u;
        uint32_t d = valid ? ((uint32_t)(key >> shift) & 255u) : 256u;
        for (int k = 0; k < 8; k++) s_wc[k][t] = 0;
        __syncthreads();
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t rank = __popc(peers & lt);
        if (valid && rank == 0) s_wc[w][d] = __popc(peers);
        __syncthreads();
        uint32_t run = 0;
        for (int k = 0; k < 8; k++) {
            uint32_t c = s_wc[k][t];
            s_wc[k][t] = run;
            run += c;
        }
        __syncthreads();
        if (valid) {
            uint32_t pos = s_off[d] + s_wc[w][d] + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        s_off[t] += run;
    }
}

template <class K> static void radix_impl(K *keys, uint32_t *vals, int64_t n, int bits, Arena &A) {
    if (n <= 1 || bits <= 0) return;
    cudaStream_t s = A.stream();
    int passes = (bits + 7) / 8;
    int tiles = (int)cdiv(n, RS_TILE);
    K *k2 = A.get<K>(n);
    uint32_t *v2 = A.get<uint32_t>(n);
    uint32_t *hist = A.get<uint32_t>((int64_t)256 * tiles);
    K *ka = keys, *kb = k2;
    uint32_t *va = vals, *vb = v2;
    for (int p = 0; p < passes; p++) {
        int shift = 8 * p;
        launch_k(k_radix_hist<K>, tiles, RS_T, 0, s, ka, n, shift, hist, tiles);
        HP_LAUNCH_CHECK();
        scan_excl(reinterpret_cast<int32_t *>(hist), reinterpret_cast<int32_t *>(hist), (int64_t)256 * tiles,
                  nullptr, A);
        launch_k(k_radix_scatter<K>, tiles, RS_T, 0, s, ka, va, kb, vb, n, shift, hist, tiles);
        HP_LAUNCH_CHECK();
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        HPC(cudaMemcpyAsync(keys, ka, n * sizeof(K), cudaMemcpyDeviceToDevice, s));
        HPC(cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    }
    A.release(k2);
    A.release(v2);
    A.release(hist);
}

// ---- variants with the element count in device memory ------------------
// Grids are sized for `cap` elements; tiles past *n_dev contribute nothing.
template <class K>
__global__ void __launch_bounds__(RS_T) k_radix_hist_dev(const K *keys, const int32_t *n_dev, int shift, uint32_t *hist,
                                                         int tiles) {
    HP_KERNEL_ENTER();
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t n = *n_dev;
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_R; r++) {
        int64_t i = base + (int64_t)r * RS_T + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(uint32_t)(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * tiles + blockIdx.x] = cnt[threadIdx.x];
}

template <class K>
__global__ void __launch_bounds__(RS_T) k_radix_scatter_dev(const K *kin, const uint32_t *vin, K *kout,
                                                            uint32_t *vout, const int32_t *n_dev, int shift,
                                                            const uint32_t *offs, int tiles) {
    HP_KERNEL_ENTER();
    __shared__ uint32_t s_off[256];
    __shared__ uint32_t s_wc[8][256];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const int64_t n = *n_dev;
    s_off[t] = offs[(int64_t)t * tiles + blockIdx.x];
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_R; r++) {
        int64_t i0 = base + (int64_t)r * RS_T;
        if (i0 >= n) break;
        int64_t i = i0 + t;
        bool valid = i < n;
        K key = valid ? kin[i] : K(0);
        uint32_t val = valid ? vin[i] : 0u;
        uint32_t d = valid ? ((uint32_t)(key >> shift) & 255u) : 256u;
        for (int k = 0; k < 8; k++) s_wc[k][t] = 0;
        __syncthreads();
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t rank = __popc(peers & lt);
        if (valid && rank == 0) s_wc[w][d] = __popc(peers);
        __syncthreads();
        uint32_t run = 0;
        for (int k = 0; k < 8; k++) {
            uint32_t c = s_wc[k][t];
            s_wc[k][t] = run;
            run += c;
        }
        __syncthreads();
        if (valid) {
            uint32_t pos = s_off[d] + s_wc[w][d] + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        s_off[t] += run;
    }
}

// Single-CTA LSD radix sort in shared memory for n <= SMALL_SORT elements
// (block_radix_sort, hp_internal.cuh); this kernel wraps it for the
// device-count sort entry points.
constexpr int SS_T = 1024, SMALL_SORT = 4096;
template <class K>
__global__ void __launch_bounds__(SS_T) k_small_sort(K *keys, uint32_t *vals, const int32_t *n_dev, int passes) {
    HP_KERNEL_ENTER();
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_wc[32][256];
    __shared__ uint32_t s_hist[256 + 33];
    block_radix_sort<K>(keys, vals, *n_dev, passes, SMALL_SORT, smem, &s_wc[0][0], s_hist);
}

template <class K>
static void radix_dev_impl(K *keys, uint32_t *vals, const int32_t *n_dev, int64_t cap, int bits, Arena &A) {
    if (cap <= 1 || bits <= 0) return;
    cudaStream_t s = A.stream();
    const int passes = (bits + 7) / 8;
    if (cap <= SMALL_SORT) {
        size_t sm = (size_t)SMALL_SORT * 2 * (sizeof(K) + sizeof(uint32_t));
        prepare_kernel((const void *)k_small_sort<K>, SS_T, sm);
        launch_k(k_small_sort<K>, 1, SS_T, sm, s, keys, vals, n_dev, passes);
        HP_LAUNCH_CHECK();
        return;
    }
    const int tiles = (int)cdiv(cap, RS_TILE);
    K *k2 = A.get<K>(cap);
    uint32_t *v2 = A.get<uint32_t>(cap);
    uint32_t *hist = A.get<uint32_t>((int64_t)256 * tiles);
    K *ka = keys, *kb = k2;
    uint32_t *va = vals, *vb = v2;
    for (int p = 0; p < passes; p++) {
        launch_k(k_radix_hist_dev<K>, tiles, RS_T, 0, s, ka, n_dev, 8 * p, hist, tiles);
        HP_LAUNCH_CHECK();
        scan_excl(reinterpret_cast<int32_t *>(hist), reinterpret_cast<int32_t *>(hist), (int64_t)256 * tiles,
                  nullptr, A);
        launch_k(k_radix_scatter_dev<K>, tiles, RS_T, 0, s, ka, va, kb, vb, n_dev, 8 * p, hist, tiles);
        HP_LAUNCH_CHECK();
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        HPC(cudaMemcpyAsync(keys, ka, cap * sizeof(K), cudaMemcpyDeviceToDevice, s));
        HPC(cudaMemcpyAsync(vals, va, cap * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    }
    A.release(k2);
    A.release(v2);
    A.release(hist);
}

void radix_sort_dev(uint32_t *keys, uint32_t *vals, const int32_t *n_dev, int64_t cap, int bits, Arena &A) {
    radix_dev_impl<uint32_t>(keys, vals, n_dev, cap, bits > 32 ? 32 : bits, A);
}
void radix_sort_dev(uint64_t *keys, uint32_t *vals, const int32_t *n_dev, int64_t cap, int bits, Arena &A) {
    radix_dev_impl<uint64_t>(keys, vals, n_dev, cap, bits > 64 ? 64 : bits, A);
}

void radix_sort(uint32_t *keys, uint32_t *vals, int64_t n, int bits, Arena &A) {
    radix_impl<uint32_t>(keys, vals, n, bits > 32 ? 32 : bits, A);
}
void radix_sort(uint64_t *keys, uint32_t *vals, int64_t n, int bits, Arena &A) {
    radix_impl<uint64_t>(keys, vals, n, bits > 64 ? 64 : bits, A);
}

}  // namespace hp
