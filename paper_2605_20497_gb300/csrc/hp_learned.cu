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
#include <cmath>
#include <vector>

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

// The sixteen feature bytes of the mutual pair (v, m), v's j-th candidate and
// m's rm-th, from the shared and inbound-shared hyperedge counts.
__device__ __forceinline__ uint4 pair_feature_bytes(const LearnIn &X, int64_t p, int32_t v, int32_t m, int32_t j,
                                                    int32_t rm, int64_t shared, int64_t inter) {
    const int32_t dv = X.ioff[v + 1] - X.ioff[v], dm = X.ioff[m + 1] - X.ioff[m];
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
    return make_uint4(f0 | f1 << 8 | f2 << 16 | f3 << 24, f4 | f5 << 8 | f6 << 16 | f7 << 24,
                      f8 | f9 << 8 | f10 << 16 | f11 << 24, f12 | f13 << 8 | f14 << 16 | f15 << 24);
}

// position of v in the list of its j-th candidate m (-1: not mutual, or no candidate)
__device__ __forceinline__ int32_t mutual_rank(const LearnIn &X, int32_t v, int32_t m) {
    if (m < 0) return -1;
    const int32_t *lm = X.candK + (int64_t)m * X.K;
    for (int32_t i = 0; i < X.K; i++)
        if (lm[i] == v) return i;
    return -1;
}

// one listed pair (v, j) by one thread: its rank and, when mutual, its
// features from the shorter incidence list searched in the other's sorted
// in- and out-halves (zero bytes unless mutual)
__device__ void merge_feats_pair(const LearnIn &X, int64_t q) {
    const int64_t p = (int64_t)X.v0 * X.K + q;   // the pair; q its row in this pass
    const int32_t v = (int32_t)(p / X.K), j = (int32_t)(p % X.K);
    const int32_t m = X.candK[p];
    const int32_t rm = mutual_rank(X, v, m);
    uint4 f = make_uint4(0, 0, 0, 0);
    if (rm >= 0) {
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
        f = pair_feature_bytes(X, p, v, m, j, rm, shared, inter);
    }
    reinterpret_cast<uint4 *>(X.feat)[q] = f;
    X.rank[q] = rm;
}

// one thread per listed pair (the whole level, or the nodes of a pass)
__global__ void k_merge_feats(LearnIn X) {
    HP_KERNEL_ENTER();
    GRID_STRIDE(q, (int64_t)(X.v1 - X.v0) * X.K) merge_feats_pair(X, q);
}

// One warp per node v: v's incidence list is staged in shared memory, and
// for each mutual candidate m the lanes walk m's list (coalesced) and look
// each hyperedge up in v's sorted in- and out-halves there.  The counts are
// the same set intersections as above.  A node whose list exceeds the
// staging area takes the one-thread-per-pair form.
constexpr int MF_T = 256, MF_CAP = 512;
__global__ void __launch_bounds__(MF_T) k_merge_feats_node(LearnIn X) {
    HP_KERNEL_ENTER();
    __shared__ int32_t s_inc[MF_T / 32][MF_CAP];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t *mine = s_inc[wid];
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = gw; u < X.v1 - X.v0; u += nw) {
        const int32_t v = X.v0 + (int32_t)u;
        const int32_t v0i = X.ioff[v], dv = X.ioff[v + 1] - v0i, niv = X.nin[v];
        if (dv > MF_CAP) {
            for (int32_t j = lane; j < X.K; j += 32) merge_feats_pair(X, u * X.K + j);
            continue;
        }
        for (int32_t t = lane; t < dv; t += 32) mine[t] = X.inc[v0i + t];
        __syncwarp();
        for (int32_t j = 0; j < X.K; j++) {
            const int64_t q = u * X.K + j, p = (int64_t)v * X.K + j;
            const int32_t m = X.candK[p];
            // v's position in m's list: lane i checks entry i
            int32_t rm = -1;
            if (m >= 0) {
                const bool hit = lane < X.K && X.candK[(int64_t)m * X.K + lane] == v;
                const unsigned bal = __ballot_sync(FULL, hit);
                rm = bal ? __ffs(bal) - 1 : -1;
            }
            uint4 f = make_uint4(0, 0, 0, 0);
            if (rm >= 0) {
                const int32_t m0 = X.ioff[m], dm = X.ioff[m + 1] - m0, nim = X.nin[m];
                int32_t sh = 0, in = 0;
                for (int32_t t = lane; t < dm; t += 32) {
                    const int32_t e = X.inc[m0 + t];
                    if (sorted_has(mine, niv, e)) {
                        sh++;
                        if (t < nim) in++;
                    } else if (sorted_has(mine + niv, dv - niv, e)) {
                        sh++;
                    }
                }
                sh = __reduce_add_sync(FULL, sh);
                in = __reduce_add_sync(FULL, in);
                f = pair_feature_bytes(X, p, v, m, j, rm, sh, in);
            }
            if (lane == 0) {
                reinterpret_cast<uint4 *>(X.feat)[q] = f;
                X.rank[q] = rm;
            }
        }
        __syncwarp();
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
    HP_KERNEL_ENTER();
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

// one thread per node of the pass: C(n) = the top Pi mutual candidates by (s, eta, id)
__global__ void k_merge_select(LearnIn X) {
    HP_KERNEL_ENTER();
    GRID_STRIDE(v0, (int64_t)(X.v1 - X.v0)) {
        const int64_t v = X.v0 + v0;
        int32_t c[16], sc[16];
        uint64_t et[16];
        int32_t have = 0;
        for (int32_t j = 0; j < X.K; j++) {
            const int64_t p = v * X.K + j, q = v0 * X.K + j;   // the pair; its row in this pass
            const int32_t m = X.candK[p];
            if (m < 0) break;
            if (X.rank[q] < 0) continue;
            const int32_t s = X.score[q];
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

// ---------------------------------------------------------------- training
// The trainable form: the same network in fp32 on features scaled by 1/256
// (z1 = W1 x + b1, h1 = relu(z1), z2 = W2 h1 + b2, h2 = relu(z2),
// o = w3 . h2 + b3), loss = mean binary cross-entropy of sigmoid(o).
// Parameters, one flat array: W1[64][16], b1[64], W2[64][64], b2[64], w3[64], b3.
constexpr int NPAR = HP_MERGE_NPARAM;
constexpr int P_W1 = 0, P_B1 = 1024, P_W2 = 1088, P_B2 = 5184, P_W3 = 5248, P_B3 = 5312;
static_assert(P_B3 + 1 == NPAR, "parameter layout");
constexpr int GRAD_CTAS = 256;   // fixed: the reduction order does not depend on the GPU
constexpr int GRAD_W = 8;        // warps per CTA, 16 rows each
constexpr int GRAD_T = GRAD_W * 32;
constexpr int GRAD_R = GRAD_W * 16;   // rows per tile
constexpr int GR_W = GRAD_R / 2 + 4;  // words per row of the transposed bf16 tiles (pairs along rows, padded)

// bf16 bits of x, rounded to nearest (ties to even)
__device__ __forceinline__ uint32_t bf16_rn(float x) {
    const uint32_t u = __float_as_uint(x);
    return (u + 0x7FFFu + ((u >> 16) & 1u)) >> 16;
}
__device__ __forceinline__ uint32_t pack2_rn(float lo, float hi) { return bf16_rn(lo) | (bf16_rn(hi) << 16); }

struct GradSmem {
    uint32_t w1[64 * 8];            // W1[j][i pair], bf16
    uint32_t w2[64 * W2_STRIDE];    // W2[k][j pair], bf16 (layer 2: B fragments over j)
    uint32_t w2t[64 * W2_STRIDE];   // W2[k][j] transposed: [j][k pair] (back-propagation: B over k)
    float b1[64], b2[64], w3[64];
    // the tile's operands of the weight gradients, transposed: [column][row pair]
    uint32_t d2t[64 * GR_W], h1t[64 * GR_W], d1t[64 * GR_W], xt[16 * GR_W];
    double loss[GRAD_W];
};

// The training step on the tensor cores.  Per tile of 128 rows, each warp
// takes 16 rows: layer 1 (8 MMAs m16n8k16, bf16 in, fp32 accumulate), layer 2
// with the clamped layer-1 accumulators as its A operand (32 MMAs), the
// output and dL/do on the CUDA cores, dL/dz1 = (dL/dz2 . W2) o [z1 > 0]
// (32 MMAs, dL/dz2 again straight from the accumulator layout); then the CTA
// forms dW2 = dz2^T h1 and dW1 = dz1^T x over the tile's rows from shared
// memory (32 + 8 MMAs over 8 warps).  Operands are rounded to bf16: W1, W2,
// h1, dL/dz2, dL/dz1 (x = f/256 is exact).  Bias, w3 and b3 gradients are
// fp32 sums.  One CTA takes a contiguous range of rows; its sums go to its
// own slot of `partial`, summed later in CTA order.
//
// m16n8k16 fragments (g = lane / 4, t = lane % 4):
//   A regs: (row g, k 2t..2t+1), (row g+8, k 2t..), (row g, k 2t+8..), (row g+8, k 2t+8..)
//   B regs: (k 2t..2t+1, col g), (k 2t+8..2t+9, col g)
//   C/D:    (row g, col 2t), (row g, col 2t+1), (row g+8, col 2t), (row g+8, col 2t+1)
__global__ void __launch_bounds__(GRAD_T) k_merge_grad(const uint8_t *feat, const float *label, int64_t count,
                                                        const float *params, float *partial, double *loss_part) {
    HP_KERNEL_ENTER();
    extern __shared__ __align__(16) unsigned char grad_smem[];
    GradSmem &S = *reinterpret_cast<GradSmem *>(grad_smem);
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, g = lane >> 2, t = lane & 3;
    for (int i = tid; i < 64 * 8; i += GRAD_T) {
        const int j = i >> 3, q = i & 7;
        S.w1[i] = pack2_rn(params[P_W1 + j * 16 + 2 * q], params[P_W1 + j * 16 + 2 * q + 1]);
    }
    for (int i = tid; i < 64 * 32; i += GRAD_T) {
        const int k = i >> 5, q = i & 31;
        S.w2[k * W2_STRIDE + q] = pack2_rn(params[P_W2 + k * 64 + 2 * q], params[P_W2 + k * 64 + 2 * q + 1]);
        // transposed: row j = k here, pairs of W2 rows 2q, 2q+1 at column j
        S.w2t[k * W2_STRIDE + q] = pack2_rn(params[P_W2 + (2 * q) * 64 + k], params[P_W2 + (2 * q + 1) * 64 + k]);
    }
    for (int i = tid; i < 64; i += GRAD_T) {
        S.b1[i] = params[P_B1 + i];
        S.b2[i] = params[P_B2 + i];
        S.w3[i] = params[P_W3 + i];
    }
    const float b3 = params[P_B3];
    const int64_t chunk = (count + gridDim.x - 1) / gridDim.x;
    const int64_t rb = (int64_t)blockIdx.x * chunk, re = min(count, rb + chunk);
    const float inv_count = count > 0 ? 1.0f / (float)count : 0.f;
    // persistent gradient accumulators: dW2 tiles (m-tile w&3, n-tiles 4(w>>2)..+3), one dW1 tile
    // (m-tile w&3, n-tile w>>2), and this lane's column sums of the warp's rows
    float gw2[4][4], gw1[4];
    float sb1[8][2], sb2[8][2], sw3[8][2], sb3 = 0.f;
#pragma unroll
    for (int a = 0; a < 4; a++) {
        gw1[a] = 0.f;
#pragma unroll
        for (int b = 0; b < 4; b++) gw2[a][b] = 0.f;
    }
#pragma unroll
    for (int c = 0; c < 8; c++)
#pragma unroll
        for (int e = 0; e < 2; e++) sb1[c][e] = sb2[c][e] = sw3[c][e] = 0.f;
    double loss = 0.0;
    __syncthreads();
    for (int64_t r0 = rb; r0 < re; r0 += GRAD_R) {
        const int64_t rw = r0 + 16 * w;   // this warp's first row
        const int64_t ra = rw + g, rbb = rw + g + 8;
        const bool va = ra < re, vb = rbb < re;
        // ---- layer 1: x (16x16, exact bf16 of f/256) . W1^T
        uint32_t xa[4];
        {
            const uint8_t *fa = feat + ra * 16, *fb = feat + rbb * 16;
            auto xv = [&](const uint8_t *f, bool ok, int i) { return ok ? (float)f[i] * (1.0f / 256.0f) : 0.f; };
            xa[0] = pack2_rn(xv(fa, va, 2 * t), xv(fa, va, 2 * t + 1));
            xa[1] = pack2_rn(xv(fb, vb, 2 * t), xv(fb, vb, 2 * t + 1));
            xa[2] = pack2_rn(xv(fa, va, 2 * t + 8), xv(fa, va, 2 * t + 9));
            xa[3] = pack2_rn(xv(fb, vb, 2 * t + 8), xv(fb, vb, 2 * t + 9));
            // x transposed for dW1: column i, rows in pairs
            const int rl = 16 * w + g;   // local row of ra (rbb = rl + 8)
            const uint32_t *xh = xa;
            // element (row, i) of the tile -> xt[i][row]; written as 16-bit halves
            uint16_t *xt16 = reinterpret_cast<uint16_t *>(S.xt);
            xt16[(2 * t) * (2 * GR_W) + rl] = (uint16_t)(xh[0] & 0xFFFF);
            xt16[(2 * t + 1) * (2 * GR_W) + rl] = (uint16_t)(xh[0] >> 16);
            xt16[(2 * t) * (2 * GR_W) + rl + 8] = (uint16_t)(xh[1] & 0xFFFF);
            xt16[(2 * t + 1) * (2 * GR_W) + rl + 8] = (uint16_t)(xh[1] >> 16);
            xt16[(2 * t + 8) * (2 * GR_W) + rl] = (uint16_t)(xh[2] & 0xFFFF);
            xt16[(2 * t + 9) * (2 * GR_W) + rl] = (uint16_t)(xh[2] >> 16);
            xt16[(2 * t + 8) * (2 * GR_W) + rl + 8] = (uint16_t)(xh[3] & 0xFFFF);
            xt16[(2 * t + 9) * (2 * GR_W) + rl + 8] = (uint16_t)(xh[3] >> 16);
        }
        float z1[8][4];
#pragma unroll
        for (int c = 0; c < 8; c++) {
            const float bl = S.b1[8 * c + 2 * t], bh = S.b1[8 * c + 2 * t + 1];
            z1[c][0] = bl;
            z1[c][1] = bh;
            z1[c][2] = bl;
            z1[c][3] = bh;
            const uint32_t *wr = S.w1 + (8 * c + g) * 8;
            mma_16816(z1[c], xa[0], xa[1], xa[2], xa[3], wr[t], wr[t + 4]);
        }
        // ---- layer 2: relu(z1) as the A operand, bf16
        float z2[8][4];
#pragma unroll
        for (int c = 0; c < 8; c++) {
            const float bl = S.b2[8 * c + 2 * t], bh = S.b2[8 * c + 2 * t + 1];
            z2[c][0] = bl;
            z2[c][1] = bh;
            z2[c][2] = bl;
            z2[c][3] = bh;
        }
#pragma unroll
        for (int kc = 0; kc < 4; kc++) {
            const float *u = z1[2 * kc], *v = z1[2 * kc + 1];
            const uint32_t a0 = pack2_rn(fmaxf(u[0], 0.f), fmaxf(u[1], 0.f)), a1 = pack2_rn(fmaxf(u[2], 0.f), fmaxf(u[3], 0.f));
            const uint32_t a2 = pack2_rn(fmaxf(v[0], 0.f), fmaxf(v[1], 0.f)), a3 = pack2_rn(fmaxf(v[2], 0.f), fmaxf(v[3], 0.f));
#pragma unroll
            for (int c = 0; c < 8; c++) {
                const uint32_t *wr = S.w2 + (8 * c + g) * W2_STRIDE + 8 * kc;
                mma_16816(z2[c], a0, a1, a2, a3, wr[t], wr[t + 4]);
            }
        }
        // ---- output, dL/do (rows g and g+8; the row's four lanes share it)
        float oa = 0.f, ob = 0.f;
#pragma unroll
        for (int c = 0; c < 8; c++) {
            const float wl = S.w3[8 * c + 2 * t], wh = S.w3[8 * c + 2 * t + 1];
            oa = fmaf(wl, fmaxf(z2[c][0], 0.f), fmaf(wh, fmaxf(z2[c][1], 0.f), oa));
            ob = fmaf(wl, fmaxf(z2[c][2], 0.f), fmaf(wh, fmaxf(z2[c][3], 0.f), ob));
        }
        oa += __shfl_xor_sync(0xffffffffu, oa, 1);
        oa += __shfl_xor_sync(0xffffffffu, oa, 2);
        ob += __shfl_xor_sync(0xffffffffu, ob, 1);
        ob += __shfl_xor_sync(0xffffffffu, ob, 2);
        oa += b3;
        ob += b3;
        float da = 0.f, db = 0.f;
        if (va) {
            const float y = label[ra];
            if (t == 0) loss += (double)(fmaxf(oa, 0.f) - oa * y + log1pf(expf(-fabsf(oa))));
            da = (1.0f / (1.0f + expf(-oa)) - y) * inv_count;
        }
        if (vb) {
            const float y = label[rbb];
            if (t == 0) loss += (double)(fmaxf(ob, 0.f) - ob * y + log1pf(expf(-fabsf(ob))));
            db = (1.0f / (1.0f + expf(-ob)) - y) * inv_count;
        }
        if (t == 0) sb3 += da + db;
        // ---- dL/dz2 = dL/do * w3 o [z2 > 0] (accumulator layout); dL/dz1 = (dz2 . W2) o [z1 > 0]
        float d2[8][4];
#pragma unroll
        for (int c = 0; c < 8; c++) {
            const float wl = S.w3[8 * c + 2 * t], wh = S.w3[8 * c + 2 * t + 1];
            d2[c][0] = z2[c][0] > 0.f ? da * wl : 0.f;
            d2[c][1] = z2[c][1] > 0.f ? da * wh : 0.f;
            d2[c][2] = z2[c][2] > 0.f ? db * wl : 0.f;
            d2[c][3] = z2[c][3] > 0.f ? db * wh : 0.f;
            sb2[c][0] += d2[c][0] + d2[c][2];
            sb2[c][1] += d2[c][1] + d2[c][3];
            sw3[c][0] += da * fmaxf(z2[c][0], 0.f) + db * fmaxf(z2[c][2], 0.f);
            sw3[c][1] += da * fmaxf(z2[c][1], 0.f) + db * fmaxf(z2[c][3], 0.f);
        }
        float d1[8][4];
#pragma unroll
        for (int c = 0; c < 8; c++) d1[c][0] = d1[c][1] = d1[c][2] = d1[c][3] = 0.f;
#pragma unroll
        for (int kc = 0; kc < 4; kc++) {
            const float *u = d2[2 * kc], *v = d2[2 * kc + 1];
            const uint32_t a0 = pack2_rn(u[0], u[1]), a1 = pack2_rn(u[2], u[3]);
            const uint32_t a2 = pack2_rn(v[0], v[1]), a3 = pack2_rn(v[2], v[3]);
#pragma unroll
            for (int c = 0; c < 8; c++) {
                const uint32_t *wr = S.w2t + (8 * c + g) * W2_STRIDE + 8 * kc;
                mma_16816(d1[c], a0, a1, a2, a3, wr[t], wr[t + 4]);
            }
        }
        // the operands of the weight gradients, transposed into shared memory
        {
            const int rl = 16 * w + g;
            uint16_t *d2t = reinterpret_cast<uint16_t *>(S.d2t), *h1t = reinterpret_cast<uint16_t *>(S.h1t),
                     *d1t = reinterpret_cast<uint16_t *>(S.d1t);
#pragma unroll
            for (int c = 0; c < 8; c++) {
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    const int col = 8 * c + 2 * t + (e & 1), row = rl + ((e & 2) ? 8 : 0);
                    const float m1 = z1[c][e] > 0.f ? 1.f : 0.f;
                    d1[c][e] *= m1;
                    d2t[col * (2 * GR_W) + row] = (uint16_t)bf16_rn(d2[c][e]);
                    h1t[col * (2 * GR_W) + row] = (uint16_t)bf16_rn(fmaxf(z1[c][e], 0.f));
                    d1t[col * (2 * GR_W) + row] = (uint16_t)bf16_rn(d1[c][e]);
                }
                sb1[c][0] += d1[c][0] + d1[c][2];
                sb1[c][1] += d1[c][1] + d1[c][3];
            }
        }
        __syncthreads();
        // ---- dW2[k][j] += sum_r dz2[r][k] h1[r][j]: warp w owns m-tile (k) w&3, n-tiles (j) 4(w>>2)..+3
        {
            const int mt = w & 3, nt0 = 4 * (w >> 2);
#pragma unroll
            for (int ks = 0; ks < GRAD_R / 16; ks++) {
                const uint32_t *ar0 = S.d2t + (16 * mt + g) * GR_W + 8 * ks, *ar1 = ar0 + 8 * GR_W;
                const uint32_t a0 = ar0[t], a1 = ar1[t], a2 = ar0[t + 4], a3 = ar1[t + 4];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const uint32_t *br = S.h1t + (8 * (nt0 + q) + g) * GR_W + 8 * ks;
                    mma_16816(gw2[q], a0, a1, a2, a3, br[t], br[t + 4]);
                }
            }
            // dW1[j][i] += sum_r dz1[r][j] x[r][i]: m-tile (j) w&3, n-tile (i) w>>2
#pragma unroll
            for (int ks = 0; ks < GRAD_R / 16; ks++) {
                const uint32_t *ar0 = S.d1t + (16 * mt + g) * GR_W + 8 * ks, *ar1 = ar0 + 8 * GR_W;
                const uint32_t *br = S.xt + (8 * (w >> 2) + g) * GR_W + 8 * ks;
                mma_16816(gw1, ar0[t], ar1[t], ar0[t + 4], ar1[t + 4], br[t], br[t + 4]);
            }
        }
        __syncthreads();
    }
    // ---- this CTA's sums into its slot, in a fixed order
    float *pp = partial + (int64_t)blockIdx.x * NPAR;
    {
        const int mt = w & 3, nt0 = 4 * (w >> 2);
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int k0 = 16 * mt + g, j0 = 8 * (nt0 + q) + 2 * t;
            pp[P_W2 + k0 * 64 + j0] = gw2[q][0];
            pp[P_W2 + k0 * 64 + j0 + 1] = gw2[q][1];
            pp[P_W2 + (k0 + 8) * 64 + j0] = gw2[q][2];
            pp[P_W2 + (k0 + 8) * 64 + j0 + 1] = gw2[q][3];
        }
        const int j0 = 16 * mt + g, i0 = 8 * (w >> 2) + 2 * t;
        pp[P_W1 + j0 * 16 + i0] = gw1[0];
        pp[P_W1 + j0 * 16 + i0 + 1] = gw1[1];
        pp[P_W1 + (j0 + 8) * 16 + i0] = gw1[2];
        pp[P_W1 + (j0 + 8) * 16 + i0 + 1] = gw1[3];
    }
    // column sums: over the 8 lanes of equal t (the warp's rows), then over the warps in order
    float *colsum = reinterpret_cast<float *>(S.d2t);   // [warp][3 * 64 + 1] scratch
#pragma unroll
    for (int c = 0; c < 8; c++)
#pragma unroll
        for (int e = 0; e < 2; e++)
#pragma unroll
            for (int o = 4; o < 32; o <<= 1) {
                sb1[c][e] += __shfl_xor_sync(0xffffffffu, sb1[c][e], o);
                sb2[c][e] += __shfl_xor_sync(0xffffffffu, sb2[c][e], o);
                sw3[c][e] += __shfl_xor_sync(0xffffffffu, sw3[c][e], o);
            }
    if (g == 0) {
#pragma unroll
        for (int c = 0; c < 8; c++)
#pragma unroll
            for (int e = 0; e < 2; e++) {
                const int col = 8 * c + 2 * t + e;
                colsum[w * 193 + col] = sb1[c][e];
                colsum[w * 193 + 64 + col] = sb2[c][e];
                colsum[w * 193 + 128 + col] = sw3[c][e];
            }
    }
    for (int o = 4; o < 32; o <<= 1) sb3 += __shfl_xor_sync(0xffffffffu, sb3, o);
    if (lane == 0) colsum[w * 193 + 192] = sb3;
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_down_sync(0xffffffffu, loss, o);
    if (lane == 0) S.loss[w] = loss;
    __syncthreads();
    if (tid < 193) {
        float a = 0.f;
        for (int ww = 0; ww < GRAD_W; ww++) a += colsum[ww * 193 + tid];
        const int at = tid < 64 ? P_B1 + tid : tid < 128 ? P_B2 + tid - 64 : tid < 192 ? P_W3 + tid - 128 : P_B3;
        pp[at] = a;
    }
    if (tid == 0) {
        double tl = 0.0;
        for (int ww = 0; ww < GRAD_W; ww++) tl += S.loss[ww];
        loss_part[blockIdx.x] = tl;
    }
}

// the CTAs' partial gradients summed in CTA order (deterministic)
__global__ void k_merge_grad_sum(const float *partial, const double *loss_part, int64_t count, float *grad,
                                 double *loss) {
    HP_KERNEL_ENTER();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < NPAR) {
        float a = 0.f;
        for (int c = 0; c < GRAD_CTAS; c++) a += partial[(int64_t)c * NPAR + i];
        grad[i] = a;
    }
    if (i == 0) {
        double t = 0.0;
        for (int c = 0; c < GRAD_CTAS; c++) t += loss_part[c];
        *loss = count > 0 ? t / (double)count : 0.0;
    }
}

// AdamW: m, v moments; c1 = 1 - beta1^t, c2 = 1 - beta2^t
__global__ void k_merge_adam(float *p, const float *g, float *m, float *v, float lr, float b1, float b2, float eps,
                             float wd, float c1, float c2) {
    HP_KERNEL_ENTER();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPAR) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / c1, vh = vi / c2;
    p[i] -= lr * (mh / (sqrtf(vh) + eps) + wd * p[i]);
}

double merge_grad(const uint8_t *feat, const float *label, int64_t count, const float *params, float *grad,
                  Arena &A) {
    cudaStream_t s = A.stream();
    float *partial = A.get<float>((int64_t)GRAD_CTAS * NPAR);
    double *lp = A.get<double>(GRAD_CTAS + 1);
    prepare_kernel((const void *)k_merge_grad, GRAD_T, sizeof(GradSmem));
    launch_k(k_merge_grad, GRAD_CTAS, GRAD_T, sizeof(GradSmem), s, feat, label, count, params, partial, lp);
    HP_LAUNCH_CHECK();
    launch_k(k_merge_grad_sum, (NPAR + 255) / 256, 256, 0, s, partial, lp, count, grad, lp + GRAD_CTAS);
    HP_LAUNCH_CHECK();
    const double loss = fetch<double>(lp + GRAD_CTAS, s);
    A.release(partial);
    A.release(lp);
    return loss;
}

void merge_adam(float *p, const float *g, float *m, float *v, int64_t step, float lr, float b1, float b2, float eps,
                float wd, cudaStream_t s) {
    const float c1 = (float)(1.0 - std::pow((double)b1, (double)step));
    const float c2 = (float)(1.0 - std::pow((double)b2, (double)step));
    launch_k(k_merge_adam, (NPAR + 255) / 256, 256, 0, s, p, g, m, v, lr, b1, b2, eps, wd, c1, c2);
    HP_LAUNCH_CHECK();
}

// Integer model of trained parameters.  With x = f / 256 and a layer's
// weights scaled by alpha (largest magnitude -> 127), the integer
// pre-activation is kappa times the float one (kappa = 256 alpha for layer 1,
// alpha / c for the next, c being the float value of one activation code of
// the layer below); the shift keeps the calibration rows' largest
// activation within 255.
void merge_quantize(const float *P, const uint8_t *calib, int64_t count, hp_merge_model &M) {
    auto alpha_of = [](const float *w, int k) {
        double m = 0.0;
        for (int i = 0; i < k; i++) m = std::max(m, (double)std::fabs(w[i]));
        return m > 0.0 ? 127.0 / m : 1.0;
    };
    auto code = [](double x) { return (int8_t)std::max(-127.0, std::min(127.0, std::nearbyint(x))); };
    auto bias = [](double x) {
        const double lim = (double)(1 << 30);
        return (int32_t)std::max(-lim, std::min(lim, std::nearbyint(x)));
    };
    auto shift_for = [](int64_t hmax) {
        int sft = 0;
        while (sft < 30 && (hmax >> sft) > 255) sft++;
        return sft;
    };
    const double a1 = alpha_of(P + P_W1, 1024), k1 = 256.0 * a1;
    for (int j = 0; j < 64; j++) {
        for (int i = 0; i < 16; i++) M.w1[j][i] = code(P[P_W1 + j * 16 + i] * a1);
        M.b1[j] = bias(P[P_B1 + j] * k1);
    }
    std::vector<int32_t> act1((size_t)count * 64);
    int64_t hmax = 0;
    for (int64_t r = 0; r < count; r++)
        for (int j = 0; j < 64; j++) {
            int64_t h = M.b1[j];
            for (int i = 0; i < 16; i++) h += (int64_t)M.w1[j][i] * calib[r * 16 + i];
            hmax = std::max(hmax, h);
            act1[(size_t)r * 64 + j] = (int32_t)std::max<int64_t>(h, 0);
        }
    M.shift1 = shift_for(hmax);
    for (auto &h : act1) h = std::min<int32_t>(255, h >> M.shift1);
    const double c1 = std::ldexp(1.0, M.shift1) / k1;
    const double a2 = alpha_of(P + P_W2, 4096), k2 = a2 / c1;
    for (int k = 0; k < 64; k++) {
        for (int j = 0; j < 64; j++) M.w2[k][j] = code(P[P_W2 + k * 64 + j] * a2);
        M.b2[k] = bias(P[P_B2 + k] * k2);
    }
    hmax = 0;
    for (int64_t r = 0; r < count; r++)
        for (int k = 0; k < 64; k++) {
            int64_t h = M.b2[k];
            for (int j = 0; j < 64; j++) h += (int64_t)M.w2[k][j] * act1[(size_t)r * 64 + j];
            hmax = std::max(hmax, h);
        }
    M.shift2 = shift_for(hmax);
    const double c2 = std::ldexp(1.0, M.shift2) / k2;
    const double a3 = alpha_of(P + P_W3, 64), k3 = a3 / c2;
    for (int k = 0; k < 64; k++) M.w3[k] = code(P[P_W3 + k] * a3);
    M.b3 = bias(P[P_B3] * k3);
}

// ---------------------------------------------------------------- host
void merge_features(const LearnIn &X, cudaStream_t s) {
    if (X.n <= 0) return;
    LearnIn Y = X;
    Y.v0 = 0;
    Y.v1 = X.n;
    launch_k(k_merge_feats, grid_for((int64_t)X.n * X.K, 256), 256, 0, s, Y);
    HP_LAUNCH_CHECK();
}

void merge_scores(const uint8_t *feat, int64_t count, const hp_merge_model *dmodel, int32_t *out, cudaStream_t s) {
    if (count <= 0) return;
    const int64_t tiles = cdiv(count, 16);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(tiles, MLP_WARPS), (int64_t)num_sms() * 8));
    launch_k(k_merge_mlp, grid, MLP_WARPS * 32, 0, s, feat, count, dmodel, out);
    HP_LAUNCH_CHECK();
}

// Node-batched (the memory remedy of Sec. VII-C applied to this design's
// per-pair rows): each pass extracts the features of `batch` nodes' listed
// pairs, scores them and selects those nodes' C(n); the mutual check reads
// the complete top-K lists, so the result does not depend on the batch.
void learned_candidates(LearnIn X, int32_t batch, cudaStream_t s) {
    if (X.n <= 0) return;
    const int32_t B = batch > 0 && batch < X.n ? batch : X.n;
    for (int32_t v0 = 0; v0 < X.n; v0 += B) {
        X.v0 = v0;
        X.v1 = std::min<int64_t>((int64_t)v0 + B, X.n);
        const int64_t pairs = (int64_t)(X.v1 - X.v0) * X.K;
        launch_k(k_merge_feats_node, grid_for((int64_t)(X.v1 - X.v0) * 32, MF_T), MF_T, 0, s, X);
        HP_LAUNCH_CHECK();
        merge_scores(X.feat, pairs, X.model, X.score, s);
        launch_k(k_merge_select, grid_for(X.v1 - X.v0, 128), 128, 0, s, X);
        HP_LAUNCH_CHECK();
    }
}

}  // namespace hp
