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
#include <atomic>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "hp_internal.cuh"

namespace hp {
void set_last_error(const std::string &msg);
}

extern "C" hp_status hp_partition_batch(const hp_instance *inst, int32_t count, const hp_options *opt,
                                        int32_t concurrency, hp_stats *stats_out, int32_t *status_out,
                                        void *stream) {
    using namespace hp;
    try {
        set_last_error("");
        if (count < 0 || (count > 0 && !inst) || concurrency < 1 || concurrency > 64) {
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
        const int W = std::min<int32_t>(concurrency, count);
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
        std::atomic<int32_t> next{0};
        std::vector<int32_t> st(count, HP_OK);
        std::vector<std::string> msg(count);
        auto work = [&](int w) {
            cudaSetDevice(dev);
            for (;;) {
                const int32_t k = next.fetch_add(1);
                if (k >= count) break;
                const int32_t i = order[k];
                const hp_instance &x = inst[i];
                hp_stats sx{};
                const hp_status r = hp_partition(x.pins, x.offsets, x.num_hedges, x.num_nodes, x.src_counts,
                                                 x.weights, x.omega, x.delta, x.seed, opt, x.part_out, &sx, ss[w]);
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
