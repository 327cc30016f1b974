// hp_noalloc.cu -- hp_connectivity_noalloc: the connectivity of Eq. 1 and the
// cut-net count for a given part vector, computed without allocating any
// device memory.
//
// Why it exists: hp_connectivity builds the full level-0 incidence and the
// sorted pins(p, e) lists of the refinement, which takes workspace from the
// library's memory pool (or from the allocator installed by
// hp_set_allocator).  Some callers cannot allow that at the moment they need
// the number: a caller whose allocator hook refuses requests while its own
// step is in flight, a process that has handed all free device memory to
// another pool, or a monitoring thread that must not take an allocator lock
// nor wait on one.  This entry point uses only a fixed scratch area that is
// part of the loaded library (a file-scope __device__ array), plus shared
// memory, so it never calls an allocator.
//
// Scratch: NA_HEAD 32-bit words of results and error flags, then
// NA_TABLE_SLOTS hash-table slots split into NA_REGIONS regions, one per CTA
// of the kernel that handles the largest hyperedges.  Slots hold part + 1,
// 0 = empty.  The table is all zero when the library is loaded (static
// device memory is zero-initialised) and every kernel here returns each slot
// it filled to zero before it exits, so it is zero at the start of every
// call.  The result words are zeroed by the call itself (an async memset on
// the caller's stream) before any kernel reads them.
//
// Limits and races: a hyperedge may hold at most NA_MAX_EDGE pins (half a
// region), else the call fails with HP_ERR_INVALID_ARG and leaves the
// scratch clean.  There is one scratch area per device, so calls that could
// overlap on one device (two streams, two host threads) race on it and give
// wrong results: callers serialise them.
//
// Placement: the scratch is device memory of this file's module, placed when
// the module is loaded on a device.  Under CUDA's lazy module loading that
// would be the first use of one of its kernels or of the array, possibly at
// a moment when the caller has no free device memory left.  So the
// library's main entry points (hp_partition*, hp_connectivity) and this call
// load the module on their first call on each device: they resolve the
// array's address and query each kernel here (noalloc_prepare below).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <string>

#include "hp_internal.cuh"

namespace hp {
void set_last_error(const std::string &msg);

namespace {

constexpr int NA_HEAD = 64;                    // 256 bytes of result and error words
constexpr int NA_REGIONS = 4;                  // CTAs of the large-hyperedge kernel
constexpr int NA_REGION_SLOTS = 1 << 19;       // 2 MiB of slots per region
constexpr int64_t NA_TABLE_SLOTS = (int64_t)NA_REGIONS * NA_REGION_SLOTS;
constexpr int32_t NA_MAX_EDGE = NA_REGION_SLOTS / 2;  // 262,144 pins
constexpr int NA_WARP_MAX = 256;               // pins of a hyperedge handled by one warp
constexpr int NA_WARP_SLOTS = 512;             // its shared table
constexpr int NA_CTA_MAX = 8192;               // pins of a hyperedge handled by one CTA in shared memory
constexpr int NA_CTA_SLOTS = 16384;            // its shared table (64 KiB)
constexpr int NA_T = 256;                      // threads of the warp kernel (8 warps)
constexpr int NA_BIG_T = 1024;                 // threads of the CTA kernels

// result words (64-bit values at even word indices)
enum : int { W_CONN = 0, W_CUT = 2, W_ERR = 4, W_BAD_EDGE = 5, W_LARGE = 6 };
// error bits
enum : uint32_t { NE_CSR = 1u, NE_PART = 2u, NE_WEIGHT = 4u, NE_SIZE = 8u };

__device__ __forceinline__ uint32_t na_hash(uint32_t key, uint32_t mask) { return (key * 0x9E3779B1u) & mask; }

__device__ __forceinline__ void na_flag(uint32_t *head, uint32_t bit) { atomicOr(&head[W_ERR], bit); }

// weight of e (checked by k_na_check)
__device__ __forceinline__ uint32_t na_weight(const int32_t *w, int32_t e) { return w ? (uint32_t)w[e] : 1u; }

__device__ __forceinline__ void na_add_result(uint32_t *head, uint32_t we, int32_t lam) {
    if (lam > 1) {
        atomicAdd((unsigned long long *)&head[W_CONN], (unsigned long long)we * (unsigned long long)(lam - 1));
        atomicAdd((unsigned long long *)&head[W_CUT], (unsigned long long)we);
    }
}

__host__ __device__ __forceinline__ uint32_t na_cap_for(int32_t pins) {
    uint32_t c = 32;
    while (c < 2u * (uint32_t)pins) c <<= 1;
    return c;
}

// lambda(e) of the hyperedge with pins [a, b): the group's `group` threads
// (index gt) insert part + 1 of every pin into `tab` (cap slots, a power of
// two >= 2 |e|, all zero on entry), counting first insertions in *count;
// then they return the cap slots to zero.  `sync` orders the phases.
template <class Sync>
__device__ void na_distinct(int32_t a, int32_t b, int gt, int group, const int32_t *pins, const int32_t *part,
                            int32_t num_nodes, int32_t num_parts, uint32_t *tab, uint32_t cap, uint32_t *head,
                            int32_t *count, Sync sync) {
    const uint32_t mask = cap - 1;
    for (int32_t j = a + gt; j < b; j += group) {
        const int32_t v = pins[j];
        if (v < 0 || v >= num_nodes) {
            na_flag(head, NE_CSR);
            continue;
        }
        const int32_t p = part[v];
        if (p < 0 || p >= num_parts) {
            na_flag(head, NE_PART);
            continue;
        }
        const uint32_t key = (uint32_t)p + 1u;
        uint32_t h = na_hash(key, mask);
        for (uint32_t probe = 0; probe < cap; probe++) {
            const uint32_t old = atomicCAS(&tab[h], 0u, key);
            if (old == 0u) {
                atomicAdd(count, 1);
                break;
            }
            if (old == key) break;
            h = (h + 1) & mask;
        }
    }
    sync();
    for (uint32_t h = (uint32_t)gt; h < cap; h += (uint32_t)group) tab[h] = 0u;
}

struct WarpSync {
    __device__ void operator()() const { __syncwarp(); }
};
struct BlockSync {
    __device__ void operator()() const { __syncthreads(); }
};

// offsets (strictly increasing from 0), weights and part ids; the kernels
// after it read pins only when this found the offsets sound
__global__ void k_na_check(const int32_t *off, const int32_t *w, const int32_t *part, int32_t num_hedges,
                           int32_t num_nodes, int32_t num_parts, uint32_t *head) {
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, step = (int64_t)gridDim.x * blockDim.x;
    if (t0 == 0 && off[0] != 0) na_flag(head, NE_CSR);
    for (int64_t e = t0; e < num_hedges; e += step) {
        if (off[e + 1] <= off[e]) na_flag(head, NE_CSR);
        if (w && (w[e] < 1 || w[e] > 65536)) na_flag(head, NE_WEIGHT);
    }
    for (int64_t v = t0; v < num_nodes; v += step)
        if (part[v] < 0 || part[v] >= num_parts) na_flag(head, NE_PART);
}

__device__ __forceinline__ bool na_sound(const uint32_t *head) {
    return (*(volatile const uint32_t *)&head[W_ERR] & (NE_CSR | NE_PART | NE_WEIGHT)) == 0u;
}

// hyperedges of up to NA_WARP_MAX pins, one warp each
__global__ void __launch_bounds__(NA_T) k_na_small(const int32_t *pins, const int32_t *off, const int32_t *w,
                                                   const int32_t *part, int32_t num_hedges, int32_t num_nodes,
                                                   int32_t num_parts, uint32_t *head) {
    __shared__ uint32_t s_tab[NA_T / 32][NA_WARP_SLOTS];
    __shared__ int32_t s_cnt[NA_T / 32];
    if (!na_sound(head)) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * (NA_T / 32) + wid, nw = (int64_t)gridDim.x * (NA_T / 32);
    for (uint32_t h = lane; h < NA_WARP_SLOTS; h += 32) s_tab[wid][h] = 0u;
    __syncwarp();
    for (int64_t e = gw; e < num_hedges; e += nw) {
        const int32_t a = off[e], b = off[e + 1];
        if (b - a > NA_WARP_MAX) {
            // tells k_na_large that it has work
            if (lane == 0 && b - a > NA_CTA_MAX) atomicOr(&head[W_LARGE], 1u);
            continue;
        }
        if (lane == 0) s_cnt[wid] = 0;
        __syncwarp();
        na_distinct(a, b, lane, 32, pins, part, num_nodes, num_parts, s_tab[wid], na_cap_for(b - a), head,
                    &s_cnt[wid], WarpSync());
        __syncwarp();
        if (lane == 0) na_add_result(head, na_weight(w, (int32_t)e), s_cnt[wid]);
    }
}

// hyperedges of NA_WARP_MAX+1 .. NA_CTA_MAX pins, one CTA each, shared table
__global__ void __launch_bounds__(NA_BIG_T) k_na_mid(const int32_t *pins, const int32_t *off, const int32_t *w,
                                                     const int32_t *part, int32_t num_hedges, int32_t num_nodes,
                                                     int32_t num_parts, uint32_t *head) {
    extern __shared__ uint32_t s_tab[];
    __shared__ int32_t s_cnt;
    if (!na_sound(head)) return;
    for (uint32_t h = threadIdx.x; h < NA_CTA_SLOTS; h += NA_BIG_T) s_tab[h] = 0u;
    __syncthreads();
    for (int64_t e = blockIdx.x; e < num_hedges; e += gridDim.x) {
        const int32_t a = off[e], b = off[e + 1];
        if (b - a <= NA_WARP_MAX || b - a > NA_CTA_MAX) continue;
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
        na_distinct(a, b, threadIdx.x, NA_BIG_T, pins, part, num_nodes, num_parts, s_tab, na_cap_for(b - a), head,
                    &s_cnt, BlockSync());
        __syncthreads();
        if (threadIdx.x == 0) na_add_result(head, na_weight(w, (int32_t)e), s_cnt);
        __syncthreads();
    }
}

// hyperedges of more than NA_CTA_MAX pins: NA_REGIONS CTAs, each with its
// own region of the scratch table; larger than NA_MAX_EDGE is an error.
// Returns at once unless k_na_small saw such a hyperedge; else each CTA
// reads NA_BIG_T offsets per step and walks the large hyperedges among them.
__global__ void __launch_bounds__(NA_BIG_T) k_na_large(const int32_t *pins, const int32_t *off, const int32_t *w,
                                                       const int32_t *part, int32_t num_hedges, int32_t num_nodes,
                                                       int32_t num_parts, uint32_t *head, uint32_t *table) {
    __shared__ int32_t s_cnt, s_nbig;
    __shared__ int32_t s_big[NA_BIG_T];
    if (!na_sound(head) || *(volatile const uint32_t *)&head[W_LARGE] == 0u) return;
    uint32_t *tab = table + (int64_t)blockIdx.x * NA_REGION_SLOTS;
    for (int64_t base = (int64_t)blockIdx.x * NA_BIG_T; base < num_hedges; base += (int64_t)gridDim.x * NA_BIG_T) {
        if (threadIdx.x == 0) s_nbig = 0;
        __syncthreads();
        const int64_t e = base + threadIdx.x;
        if (e < num_hedges) {
            const int32_t len = off[e + 1] - off[e];
            if (len > NA_MAX_EDGE) {
                na_flag(head, NE_SIZE);
                atomicMax((int *)&head[W_BAD_EDGE], len);
            } else if (len > NA_CTA_MAX) {
                s_big[atomicAdd(&s_nbig, 1)] = (int32_t)e;
            }
        }
        __syncthreads();
        const int32_t nbig = s_nbig;
        for (int32_t k = 0; k < nbig; k++) {
            const int32_t eb = s_big[k], a = off[eb], b = off[eb + 1];
            if (threadIdx.x == 0) s_cnt = 0;
            __syncthreads();
            na_distinct(a, b, threadIdx.x, NA_BIG_T, pins, part, num_nodes, num_parts, tab, na_cap_for(b - a),
                        head, &s_cnt, BlockSync());
            __syncthreads();
            if (threadIdx.x == 0) na_add_result(head, na_weight(w, eb), s_cnt);
            __syncthreads();
        }
    }
}

}  // namespace
}  // namespace hp

// The scratch area: 256 B of result words + 8 MiB of table, one copy per
// device, zero-initialised when the module loads.
static __device__ __align__(256) uint32_t g_na_scratch[hp::NA_HEAD + hp::NA_TABLE_SLOTS];

// ------------------------------------------------------------------ C ABI
namespace {
constexpr int NA_MAX_DEVICES = 64;
std::atomic<uint32_t *> g_na_addr[NA_MAX_DEVICES];
std::mutex g_na_mu;

// Device address of the scratch on the current device, looked up once per
// device with that device current (the first lookup also loads this
// module's kernels, so the scratch is placed then).  The cached address
// belongs to the device's context: after cudaDeviceReset it is stale, so a
// process that resets a device must not call this library on it again.
uint32_t *na_scratch_of_current_device() {
    int dev = 0;
    HPC(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NA_MAX_DEVICES) throw hp::Error(HP_ERR_INTERNAL, "device index out of range");
    uint32_t *a = g_na_addr[dev].load(std::memory_order_acquire);
    if (a) return a;
    std::lock_guard<std::mutex> lk(g_na_mu);
    a = g_na_addr[dev].load(std::memory_order_relaxed);
    if (a) return a;
    void *p = nullptr;
    HPC(cudaGetSymbolAddress(&p, g_na_scratch));
    cudaFuncAttributes fa;
    for (const void *f : {(const void *)hp::k_na_check, (const void *)hp::k_na_small, (const void *)hp::k_na_mid,
                          (const void *)hp::k_na_large})
        HPC(cudaFuncGetAttributes(&fa, f));
    a = static_cast<uint32_t *>(p);
    g_na_addr[dev].store(a, std::memory_order_release);
    return a;
}
}  // namespace

namespace hp {
// called by the library's main entry points on their first call per device
void noalloc_prepare() { (void)na_scratch_of_current_device(); }
}  // namespace hp

extern "C" hp_status hp_connectivity_noalloc(const int32_t *pins, const int32_t *offsets, int32_t num_hedges,
                                             const int32_t *weights, const int32_t *part, int32_t num_nodes,
                                             int32_t num_parts, int64_t *conn_out, int64_t *cutnet_out,
                                             void *stream) {
    using namespace hp;
    try {
        set_last_error("");
        if (num_hedges < 0 || num_nodes < 0 || num_parts < 0 || !offsets || (num_nodes > 0 && !part) ||
            (num_hedges > 0 && !pins)) {
            set_last_error("invalid argument");
            return HP_ERR_INVALID_ARG;
        }
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        uint32_t *scratch = na_scratch_of_current_device();
        uint32_t *head = scratch, *table = scratch + NA_HEAD;
        HPC(cudaMemsetAsync(head, 0, NA_HEAD * sizeof(uint32_t), s));
        const int sms = num_sms();
        const int64_t items = std::max<int64_t>(num_hedges, num_nodes);
        const int cgrid = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(items, 256), (int64_t)sms * 8));
        k_na_check<<<cgrid, 256, 0, s>>>(offsets, weights, part, num_hedges, num_nodes, num_parts, head);
        HP_LAUNCH_CHECK();
        if (num_hedges > 0) {
            const int grid = (int)std::min<int64_t>(cdiv(num_hedges, NA_T / 32), (int64_t)sms * 8);
            k_na_small<<<grid, NA_T, 0, s>>>(pins, offsets, weights, part, num_hedges, num_nodes, num_parts, head);
            HP_LAUNCH_CHECK();
            const size_t sm = NA_CTA_SLOTS * sizeof(uint32_t);
            HPC(cudaFuncSetAttribute((const void *)k_na_mid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            k_na_mid<<<(int)std::min<int64_t>(num_hedges, (int64_t)sms * 2), NA_BIG_T, sm, s>>>(
                pins, offsets, weights, part, num_hedges, num_nodes, num_parts, head);
            HP_LAUNCH_CHECK();
            k_na_large<<<(int)std::min<int64_t>(num_hedges, NA_REGIONS), NA_BIG_T, 0, s>>>(
                pins, offsets, weights, part, num_hedges, num_nodes, num_parts, head, table);
            HP_LAUNCH_CHECK();
        }
        uint32_t h[8];
        HPC(cudaMemcpyAsync(h, head, sizeof h, cudaMemcpyDeviceToHost, s));
        HPC(cudaStreamSynchronize(s));
        const uint32_t err = h[W_ERR];
        if (err & NE_SIZE) {
            set_last_error("a hyperedge of " + std::to_string(h[W_BAD_EDGE]) + " pins exceeds the limit of " +
                           std::to_string(NA_MAX_EDGE) + " pins of hp_connectivity_noalloc");
            return HP_ERR_INVALID_ARG;
        }
        if (err & NE_CSR) {
            set_last_error("offsets not strictly increasing from 0, or a pin out of range");
            return HP_ERR_BAD_CSR;
        }
        if (err & (NE_PART | NE_WEIGHT)) {
            set_last_error((err & NE_PART) ? "part id out of range" : "weight outside 1..65536");
            return HP_ERR_INVALID_ARG;
        }
        uint64_t conn, cut;
        memcpy(&conn, &h[W_CONN], 8);
        memcpy(&cut, &h[W_CUT], 8);
        if (conn_out) *conn_out = (int64_t)conn;
        if (cutnet_out) *cutnet_out = (int64_t)cut;
        return HP_OK;
    } catch (const hp::Error &x) {
        set_last_error(x.what());
        return x.status;
    } catch (const std::exception &x) {
        set_last_error(x.what());
        return HP_ERR_INTERNAL;
    }
}
