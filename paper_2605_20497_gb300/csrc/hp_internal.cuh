// hp_internal.cuh -- shared declarations of the CUDA partitioner (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <stdexcept>
#include <string>
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
void fill_i32(int32_t *p, int64_t n, int32_t v, cudaStream_t s);
void iota_i32(int32_t *p, int64_t n, cudaStream_t s);

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
    int32_t *nin = nullptr;    // [n] |in(v)|
    int32_t *gamma = nullptr;  // [n] node -> node of the next level
    int32_t *nbnd = nullptr;   // [n] upper bound on |N(v)| (neighbour table sizing)
};

struct Params {
    int32_t omega, delta;
    uint64_t seed;
    hp_options o;
};

// graph construction (hp_graph.cu)
uint32_t validate_and_build_level0(const int32_t *pins, const int32_t *offsets, int32_t e, int32_t n,
                                   const int32_t *src_counts, const int32_t *weights, const Params &P, Level &L,
                                   int32_t *w_out, Arena &A);
void build_incidence(Level &L, Arena &A);
// level graph from caller arrays (device): copies them and builds the incidence
void make_level(int32_t n, int32_t e, const int32_t *off, const int32_t *pins, const int32_t *nsrc,
                const int32_t *size, Level &L, Arena &A);
void contract_level(const Level &L, const int32_t *mate, Level &C, Arena &A);

// coarsening (hp_coarsen.cu)
struct CoarsenOut {
    int64_t pairs = 0, iso_pairs = 0, pin_visits = 0, neighbours = 0;
};
// prop_events (optional): two events recorded around the proposal launches
CoarsenOut coarsen_level(Level &L, int32_t level, const int32_t *w, const Params &P, int32_t *mate, Arena &A,
                         uint32_t *err_dev, int32_t *cand_out = nullptr, uint64_t *score_out = nullptr,
                         cudaEvent_t *prop_events = nullptr);

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
};
RefineOut refine_level(const Level &L, const int32_t *w, int32_t nparts, const Params &P, int32_t *rho, Arena &A,
                       uint32_t *err_dev);
void objective(const Level &L, const int32_t *w, const int32_t *rho, int32_t nparts, int64_t *conn_dev,
               int64_t *cutnet_dev, Arena &A);
void part_stats(const Level &L, const int32_t *w, const int32_t *part, int32_t nparts, int32_t omega, int32_t delta,
                int64_t *out, Arena &A);

// allocator hook (hp_prims.cu)
void set_allocator(void *(*a)(size_t, void *), void (*f)(void *, void *), void *ctx);

}  // namespace hp
