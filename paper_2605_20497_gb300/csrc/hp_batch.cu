// hp_batch.cu -- hp_partition_batch: many independent hypergraphs in one
// call.  Small instances leave most of the GPU idle (their levels are chains
// of short kernels over a few thousand nodes), so the batch runs several of
// them at once: host worker threads, each with its own CUDA stream, take the
// instances largest first and partition each exactly as hp_partition does.
// The library is reentrant across streams and threads (per-device memory
// pools and attribute caches are locked, the result mailbox and the error
// text are per thread), so each result is the one hp_partition returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "hp_internal.cuh"

namespace hp {
void set_last_error(const std::string &msg);

// Instances of one size class run as one group: `W` host workers, one
// stream each, take them largest first.  Returns the seconds it took.
static double run_group(const hp_instance *inst, const std::vector<int32_t> &ids, int W, int dev,
                        const hp_options *opt, cudaStream_t caller, hp_stats *stats_out, std::vector<int32_t> &st,
                        std::vector<std::string> &msg) {
    using namespace hp;
    const auto t0 = std::chrono::steady_clock::now();
    W = std::max(1, std::min<int>(W, (int)ids.size()));
    std::vector<cudaStream_t> ss(W, nullptr);
    std::vector<cudaEvent_t> done(W, nullptr);
    cudaEvent_t start = nullptr;
    HPC(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
    HPC(cudaEventRecord(start, caller));
    for (int w = 0; w < W; w++) {
        HPC(cudaStreamCreateWithFlags(&ss[w], cudaStreamNonBlocking));
        HPC(cudaEventCreateWithFlags(&done[w], cudaEventDisableTiming));
        HPC(cudaStreamWaitEvent(ss[w], start, 0));
    }
    std::atomic<size_t> next{0};
    auto work = [&](int w) {
        cudaSetDevice(dev);
        t_plain_launches = true;
        for (;;) {
            const size_t k = next.fetch_add(1);
            if (k >= ids.size()) break;
            const int32_t i = ids[k];
            const hp_instance &x = inst[i];
            hp_stats sx{};
            const hp_status r = hp_partition(x.pins, x.offsets, x.num_hedges, x.num_nodes, x.src_counts, x.weights,
                                             x.omega, x.delta, x.seed, opt, x.part_out, &sx, ss[w]);
            st[i] = r;
            if (r != HP_OK) msg[i] = hp_last_error();
            if (stats_out) stats_out[i] = sx;
        }
        cudaEventRecord(done[w], ss[w]);
    };
    std::vector<std::thread> th;
    th.reserve(W);
    for (int w = 0; w < W; w++) th.emplace_back(work, w);
    for (auto &t : th) t.join();
    for (int w = 0; w < W; w++) {
        HPC(cudaStreamWaitEvent(caller, done[w], 0));
        cudaEventDestroy(done[w]);
        cudaStreamDestroy(ss[w]);
    }
    cudaEventDestroy(start);
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// size class of an instance by its nodes + hyperedges (known on the host):
// [0, 2^12), then factors of 4 up to [2^20, ...)
constexpr int BUCKETS = 6;
static int bucket_of(const hp_instance &x) {
    const int64_t units = (int64_t)x.num_nodes + x.num_hedges;
    int c = 0;
    for (int64_t lim = (int64_t)1 << 12; units >= lim && c < BUCKETS - 1; lim <<= 2) c++;
    return c;
}

// Autotuned concurrency per (device, size class), kept for later calls: the
// first instances of a class run in groups of 2c at c = 4, 8, 16, 32, 64 in
// flight, and the rest of the class (and later batches) at the c that gave
// the most pins per second.  Only the schedule is tuned: every instance is
// partitioned once, exactly as hp_partition would.
static std::mutex g_tune_mu;
static std::vector<std::array<int, BUCKETS>> g_tuned;   // per device; 0 = not tuned yet

int32_t batch_tuned_concurrency(int dev, int bucket) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (dev < 0 || dev >= (int)g_tuned.size() || bucket < 0 || bucket >= BUCKETS) return 0;
    return g_tuned[dev][bucket];
}
}  // namespace hp

extern "C" hp_status hp_partition_batch(const hp_instance *inst, int32_t count, const hp_options *opt,
                                        int32_t concurrency, hp_stats *stats_out, int32_t *status_out,
                                        void *stream) {
    using namespace hp;
    try {
        set_last_error("");
        if (count < 0 || (count > 0 && !inst) || concurrency < 0 || concurrency > 64) {
            set_last_error("invalid argument");
            return HP_ERR_INVALID_ARG;
        }
        if (count == 0) return HP_OK;
        int dev = 0;
        HPC(cudaGetDevice(&dev));
        cudaStream_t caller = static_cast<cudaStream_t>(stream);
        // largest first, so that the last instances to start are short
        std::vector<int32_t> order(count);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
            return (int64_t)inst[a].num_nodes + inst[a].num_hedges > (int64_t)inst[b].num_nodes + inst[b].num_hedges;
        });
        std::vector<int32_t> st(count, HP_OK);
        std::vector<std::string> msg(count);
        if (concurrency > 0) {
            run_group(inst, order, concurrency, dev, opt, caller, stats_out, st, msg);
        } else {
            // autotuned: size classes largest first
            std::vector<std::vector<int32_t>> cls(BUCKETS);
            std::vector<int64_t> cls_pins(BUCKETS, 0);
            for (int32_t i : order) cls[bucket_of(inst[i])].push_back(i);
            for (int b = BUCKETS - 1; b >= 0; b--) {
                std::vector<int32_t> &ids = cls[b];
                if (ids.empty()) continue;
                size_t at = 0;
                int best = batch_tuned_concurrency(dev, b);
                if (best == 0) {
                    double best_rate = -1.0;
                    for (int c : {4, 8, 16, 32, 64}) {
                        const size_t take = std::min(ids.size() - at, (size_t)(2 * c));
                        if (take == 0) break;
                        std::vector<int32_t> grp(ids.begin() + at, ids.begin() + at + take);
                        int64_t units = 0;
                        for (int32_t i : grp) units += (int64_t)inst[i].num_nodes + inst[i].num_hedges;
                        const double sec = run_group(inst, grp, c, dev, opt, caller, stats_out, st, msg);
                        HPC(cudaStreamSynchronize(caller));
                        const double rate = units / std::max(sec, 1e-9);
                        if (rate > best_rate) {
                            best_rate = rate;
                            best = c;
                        }
                        at += take;
                    }
                    if (at == ids.size() && ids.size() < 2 * 4 + 2 * 8) best = 0;   // too few to tell
                    if (best > 0) {
                        std::lock_guard<std::mutex> lk(g_tune_mu);
                        if ((int)g_tuned.size() <= dev) g_tuned.resize(dev + 1, std::array<int, BUCKETS>{});
                        g_tuned[dev][b] = best;
                    }
                }
                if (at < ids.size()) {
                    std::vector<int32_t> rest(ids.begin() + at, ids.end());
                    run_group(inst, rest, best > 0 ? best : 16, dev, opt, caller, stats_out, st, msg);
                }
            }
        }
        if (status_out) std::copy(st.begin(), st.end(), status_out);
        for (int32_t i = 0; i < count; i++) {
            if (st[i] != HP_OK) {
                set_last_error("instance " + std::to_string(i) + ": " + msg[i]);
                return static_cast<hp_status>(st[i]);
            }
        }
        return HP_OK;
    } catch (const hp::Error &x) {
        set_last_error(x.what());
        return x.status;
    } catch (const std::exception &x) {
        set_last_error(x.what());
        return HP_ERR_INTERNAL;
    }
}

extern "C" int32_t hp_batch_tuned_concurrency(int32_t device, int32_t size_class) {
    return hp::batch_tuned_concurrency(device, size_class);
}
