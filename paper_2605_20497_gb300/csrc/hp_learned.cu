// hp_learned.cu -- learned merge priority, a growth of the candidate proposal
// of Sec. V-C that the paper does not have.  Every node's top-K valid
// neighbours by (eta, id) come from the proposal kernels (K in place of Pi);
// a pair stays a candidate only when each end lists the other; C(n) is the
// top Pi of the node's candidates by (s, eta, id), s the score of a small
// integer MLP (16 -> 64 -> 64 -> 1) on sixteen symmetric pair features.  The
// matching keeps eta as its weight.  Symmetric scores over a symmetric
// candidate relation keep the proposal graph free of cycles longer than two,
// which the matching of Sec. V-D relies on.
//
// The MLP runs on the tensor cores: bf16 operands, fp32 accumulation
// (mma.sync m16n8k16).  Weight codes lie in [-127, 127] and activations in
// 0..255, so every operand is an exact bf16 and every product and partial
// sum an integer below 2^21: the fp32 accumulation is exact and the score is
// the same integer on any hardware and in any summation order.
#include <cuda_runtime.h>

#include <algorithm>

#include "hp_internal.cuh"

namespace hp {

static int grid_for(int64_t n, int block) {
    int64_t g = cdiv(n, block);
    const int64_t cap = (int64_t)num_sms() * 32;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}
#define GRID_STRIDE(i, n) \
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

bool merge_model_ok(const hp_merge_model &m) {
    auto codes_ok = [](const int8_t *w, int k) {
        for (int i = 0; i < k; i++)
            if (w[i] < -127) return false;
        return true;
    };
    auto bias_ok = [](int32_t b) { return b >= -(1 << 30) && b <= (1 << 30); };
    if (!codes_ok(&m.w1[0][0], 64 * 16) || !codes_ok(&m.w2[0][0], 64 * 64) || !codes_ok(m.w3, 64)) return false;
    for (int i = 0; i < 64; i++)
        if (!bias_ok(m.b1[i]) || !bias_ok(m.b2[i])) return false;
    return bias_ok(m.b3) && m.shift1 >= 0 && m.shift1 <= 30 && m.shift2 >= 0 && m.shift2 <= 30;
}

// ---------------------------------------------------------------- features
// 0 for 0, else min(255, 1 + 4 floor(log2 x) + the two bits after the leading one)
__device__ __forceinline__ uint32_t log_code(uint64_t x) {
    if (x == 0) return 0u;
    const int b = 63 - __clzll((long long)x);
    const uint64_t frac = b >= 2 ? (x >> (b - 2)) & 3u : (x << (2 - b)) & 3u;
    const int c = 1 + 4 * b + (int)frac;
    return (uint32_t)(c > 255 ? 255 : c);
}

__device__ __forceinline__ bool sorted_has(const int32_t *a, int32_t len, int32_t x) {
    int32_t lo = 0, hi = len;
    while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo < len && a[lo] == x;
}

// one thread per listed pair (v, j): rank = position of v in the list of its
// j-th candidate m (-1: not mutual, or no candidate), and the pair's sixteen
// feature bytes (zero unless mutual)
__global__ void k_merge_feats(LearnIn X) {
    const int64_t total = (int64_t)X.n * X.K;
    GRID_STRIDE(p, total) {
        const int32_t v = (int32_t)(p / X.K), j = (int32_t)(p % X.K);
        const int32_t m = X.candK[p];
        int32_t rm = -1;
        if (m >= 0) {
            const int32_t *lm = X.candK + (int64_t)m * X.K;
            for (int32_t i = 0; i < X.K; i++)
                if (lm[i] == v) {
                    rm = i;
                    break;
                }
        }
        uint32_t w0 = 0, w1 = 0, w2 = 0, w3 = 0;
        if (rm >= 0) {
            // walk the shorter incidence list; search the other's sorted in- and out-halves
            const int32_t dv = X.ioff[v + 1] - X.ioff[v], dm = X.ioff[m + 1] - X.ioff[m];
            const int32_t a = dv <= dm ? v : m, b = dv <= dm ? m : v;
            const int32_t a0 = X.ioff[a], a1 = X.ioff[a + 1], a_in_end = a0 + X.nin[a];
            const int32_t *b_in = X.inc + X.ioff[b];
            const int32_t nb_in = X.nin[b], nb_out = X.ioff[b + 1] - X.ioff[b] - X.nin[b];
            int64_t shared = 0, inter = 0;
            for (int32_t t = a0; t < a1; t++) {
                const int32_t e = X.inc[t];
                if (sorted_has(b_in, nb_in, e)) {
                    shared++;
                    if (t < a_in_end) inter++;
                } else if (sorted_has(b_in + nb_in, nb_out, e)) {
                    shared++;
                }
            }
            const int64_t sv = X.size[v], sm = X.size[m], iv = X.nin[v], im = X.nin[m];
            const int64_t uni = iv + im - inter;
            const uint32_t f0 = log_code(X.csK[p]);
            const uint32_t f1 = log_code((uint64_t)shared);
            const uint32_t f2 = log_code((uint64_t)inter);
            const uint32_t f3 = log_code((uint64_t)min(sv, sm)), f4 = log_code((uint64_t)max(sv, sm));
            const uint32_t f5 = log_code((uint64_t)min(iv, im)), f6 = log_code((uint64_t)max(iv, im));
            const uint32_t f7 = log_code((uint64_t)min(dv, dm)), f8 = log_code((uint64_t)max(dv, dm));
            const uint32_t f9 = (uint32_t)(255 * (sv + sm) / X.omega);
            const uint32_t f10 = X.delta > 0 ? (uint32_t)(255 * uni / X.delta) : 0u;
            const uint32_t f11 = (uint32_t)min(X.level, 255);
            const uint32_t f12 = uni > 0 ? (uint32_t)(255 * inter / uni) : 0u;
            const uint32_t f13 = (uint32_t)min(j, rm), f14 = (uint32_t)max(j, rm);
            const uint32_t f15 = log_code((uint64_t)(iv + im));
            w0 = f0 | f1 << 8 | f2 << 16 | f3 << 24;
            w1 = f4 | f5 << 8 | f6 << 16 | f7 << 24;
            w2 = f8 | f9 << 8 | f10 << 16 | f11 << 24;
            w3 = f12 | f13 << 8 | f14 << 16 | f15 << 24;
        }
        reinterpret_cast<uint4 *>(X.feat)[p] = make_uint4(w0, w1, w2, w3);
        X.rank[p] = rm;
    }
}

// ---------------------------------------------------------------- MLP
// bf16 bits of an integer of magnitude at most 256: the float has at most
// eight significant bits, so its upper half is the exact bf16
__device__ __forceinline__ uint32_t bf16_bits(int32_t x) { return __float_as_uint((float)x) >> 16; }
__device__ __forceinline__ uint32_t pack_bf16(int32_t lo, int32_t hi) { return bf16_bits(lo) | (bf16_bits(hi) << 16); }

// d += A (16x16, row) * B (16x8, col), bf16 in, fp32 accumulate
__device__ __forceinline__ void mma_16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                          uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ int32_t act_code(float acc, int32_t bias, int shift) {
    const int32_t h = __float2int_rn(acc) + bias;   // acc is an exact integer
    return h <= 0 ? 0 : min(255, h >> shift);
}

constexpr int MLP_WARPS = 8;
constexpr int W2_STRIDE = 36;   // words per row of the packed W2 (32 + 4: conflict-free fragment loads)

// One warp scores 16 feature rows per step (the M = 16 rows of the MMA).
// Fragment layout of m16n8k16 (g = lane / 4, t = lane % 4):
//   A regs: (row g, k 2t..2t+1), (row g+8, k 2t..), (row g, k 2t+8..), (row g+8, k 2t+8..)
//   B regs: (k 2t..2t+1, col g), (k 2t+8..2t+9, col g)
//   C/D:    (row g, col 2t), (row g, col 2t+1), (row g+8, col 2t), (row g+8, col 2t+1)
// so the layer-1 outputs of n-tiles 2c and 2c+1 are, as they stand in the
// registers, the A operand of layer 2 for k-chunk c.
__global__ void __launch_bounds__(MLP_WARPS * 32) k_merge_mlp(const uint8_t *feat, int64_t count,
                                                               const hp_merge_model *M, int32_t *out) {
    __shared__ uint32_t s_w1[64 * 8];           // [hidden j][feature pair]
    __shared__ uint32_t s_w2[64 * W2_STRIDE];   // [hidden k][hidden pair]
    __shared__ int32_t s_b1[64], s_b2[64], s_w3[64];
    for (int i = threadIdx.x; i < 64 * 8; i += blockDim.x) {
        const int j = i >> 3, q = i & 7;
        s_w1[i] = pack_bf16(M->w1[j][2 * q], M->w1[j][2 * q + 1]);
    }
    for (int i = threadIdx.x; i < 64 * 32; i += blockDim.x) {
        const int k = i >> 5, q = i & 31;
        s_w2[k * W2_STRIDE + q] = pack_bf16(M->w2[k][2 * q], M->w2[k][2 * q + 1]);
    }
    for (int i = threadIdx.x; i < 64; i += blockDim.x) {
        s_b1[i] = M->b1[i];
        s_b2[i] = M->b2[i];
        s_w3[i] = M->w3[i];
    }
    __syncthreads();
    const int sh1 = M->shift1, sh2 = M->shift2;
    const int32_t b3 = M->b3;
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int64_t tiles = (count + 15) / 16;
    // warp-uniform loop: all 32 lanes take part in every MMA
    for (int64_t tile = (int64_t)blockIdx.x * MLP_WARPS + (threadIdx.x >> 5); tile < tiles;
         tile += (int64_t)gridDim.x * MLP_WARPS) {
        const int64_t r0 = tile * 16 + g, r1 = r0 + 8;
        const uint8_t *f0 = feat + r0 * 16, *f1 = feat + r1 * 16;
        const bool in0 = r0 < count, in1 = r1 < count;
        const uint32_t a0 = in0 ? pack_bf16(f0[2 * t], f0[2 * t + 1]) : 0u;
        const uint32_t a1 = in1 ? pack_bf16(f1[2 * t], f1[2 * t + 1]) : 0u;
        const uint32_t a2 = in0 ? pack_bf16(f0[2 * t + 8], f0[2 * t + 9]) : 0u;
        const uint32_t a3 = in1 ? pack_bf16(f1[2 * t + 8], f1[2 * t + 9]) : 0u;
        // layer 1: eight n-tiles of 8 hidden units
        uint32_t h[4][4];   // layer-2 A fragments, one per k-chunk of 16 hidden units
#pragma unroll
        for (int c = 0; c < 4; c++) {
            int32_t x[2][4];
#pragma unroll
            for (int half = 0; half < 2; half++) {
                const int nt = 2 * c + half;
                float d[4] = {0.f, 0.f, 0.f, 0.f};
                const uint32_t *wr = s_w1 + (nt * 8 + g) * 8;
                mma_16816(d, a0, a1, a2, a3, wr[t], wr[t + 4]);
                const int col = nt * 8 + 2 * t;
                x[half][0] = act_code(d[0], s_b1[col], sh1);
                x[half][1] = act_code(d[1], s_b1[col + 1], sh1);
                x[half][2] = act_code(d[2], s_b1[col], sh1);
                x[half][3] = act_code(d[3], s_b1[col + 1], sh1);
            }
            h[c][0] = pack_bf16(x[0][0], x[0][1]);   // row g,   k 2t..2t+1
            h[c][1] = pack_bf16(x[0][2], x[0][3]);   // row g+8, k 2t..2t+1
            h[c][2] = pack_bf16(x[1][0], x[1][1]);   // row g,   k 2t+8..2t+9
            h[c][3] = pack_bf16(x[1][2], x[1][3]);   // row g+8, k 2t+8..2t+9
        }
        // layer 2 and the output dot product
        int32_t acc0 = 0, acc1 = 0;
#pragma unroll
        for (int nt = 0; nt < 8; nt++) {
            float d[4] = {0.f, 0.f, 0.f, 0.f};
            const uint32_t *wr = s_w2 + (nt * 8 + g) * W2_STRIDE;
#pragma unroll
            for (int c = 0; c < 4; c++) mma_16816(d, h[c][0], h[c][1], h[c][2], h[c][3], wr[8 * c + t], wr[8 * c + t + 4]);
            const int col = nt * 8 + 2 * t;
            acc0 += s_w3[col] * act_code(d[0], s_b2[col], sh2) + s_w3[col + 1] * act_code(d[1], s_b2[col + 1], sh2);
            acc1 += s_w3[col] * act_code(d[2], s_b2[col], sh2) + s_w3[col + 1] * act_code(d[3], s_b2[col + 1], sh2);
        }
        // the four lanes of a row group hold disjoint columns
        acc0 += __shfl_xor_sync(0xffffffffu, acc0, 1);
        acc0 += __shfl_xor_sync(0xffffffffu, acc0, 2);
        acc1 += __shfl_xor_sync(0xffffffffu, acc1, 1);
        acc1 += __shfl_xor_sync(0xffffffffu, acc1, 2);
        if (t == 0) {
            if (in0) out[r0] = b3 + acc0;
            if (in1) out[r1] = b3 + acc1;
        }
    }
}

// ---------------------------------------------------------------- selection
__device__ __forceinline__ bool learned_gt(int32_t s1, uint64_t e1, int32_t m1, int32_t s2, uint64_t e2, int32_t m2) {
    if (s1 != s2) return s1 > s2;
    return e1 > e2 || (e1 == e2 && m1 > m2);
}

// one thread per node: C(n) = the top Pi mutual candidates by (s, eta, id)
__global__ void k_merge_select(LearnIn X) {
    GRID_STRIDE(v, (int64_t)X.n) {
        int32_t c[16], sc[16];
        uint64_t et[16];
        int32_t have = 0;
        for (int32_t j = 0; j < X.K; j++) {
            const int64_t p = v * X.K + j;
            const int32_t m = X.candK[p];
            if (m < 0) break;
            if (X.rank[p] < 0) continue;
            const int32_t s = X.score[p];
            const uint64_t e = X.csK[p];
            int32_t pos = have;
            while (pos > 0 && learned_gt(s, e, m, sc[pos - 1], et[pos - 1], c[pos - 1])) pos--;
            if (pos < X.pi) {
                for (int32_t q = (have < X.pi ? have : X.pi - 1); q > pos; q--) {
                    c[q] = c[q - 1];
                    sc[q] = sc[q - 1];
                    et[q] = et[q - 1];
                }
                c[pos] = m;
                sc[pos] = s;
                et[pos] = e;
                if (have < X.pi) have++;
            }
        }
        for (int32_t r = 0; r < X.pi; r++) {
            X.cand[v * X.pi + r] = r < have ? c[r] : -1;
            X.cscore[v * X.pi + r] = r < have ? et[r] : 0ull;
        }
    }
}

// ---------------------------------------------------------------- host
void merge_scores(const uint8_t *feat, int64_t count, const hp_merge_model *dmodel, int32_t *out, cudaStream_t s) {
    if (count <= 0) return;
    const int64_t tiles = cdiv(count, 16);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(tiles, MLP_WARPS), (int64_t)num_sms() * 8));
    k_merge_mlp<<<grid, MLP_WARPS * 32, 0, s>>>(feat, count, dmodel, out);
    HP_LAUNCH_CHECK();
}

void learned_candidates(const LearnIn &X, cudaStream_t s) {
    if (X.n <= 0) return;
    const int64_t pairs = (int64_t)X.n * X.K;
    k_merge_feats<<<grid_for(pairs, 256), 256, 0, s>>>(X);
    HP_LAUNCH_CHECK();
    merge_scores(X.feat, pairs, X.model, X.score, s);
    k_merge_select<<<grid_for(X.n, 128), 128, 0, s>>>(X);
    HP_LAUNCH_CHECK();
}

}  // namespace hp
