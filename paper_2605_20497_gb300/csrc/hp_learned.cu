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

// one thread per listed pair (v, j): rank = position of v in the list of its
// j-th candidate m (-1: not mutual, or no candidate), and the pair's sixteen
// feature bytes (zero unless mutual)
__global__ void k_merge_feats(LearnIn X) {
    const int64_t base = (int64_t)X.v0 * X.K, total = (int64_t)(X.v1 - X.v0) * X.K;
    GRID_STRIDE(q, total) {
        const int64_t p = base + q;   // the pair; q its row in this pass
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
        reinterpret_cast<uint4 *>(X.feat)[q] = make_uint4(w0, w1, w2, w3);
        X.rank[q] = rm;
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

// one thread per node of the pass: C(n) = the top Pi mutual candidates by (s, eta, id)
__global__ void k_merge_select(LearnIn X) {
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
constexpr int GRAD_T = 256;
constexpr int GRAD_R = 32;       // rows per tile
constexpr int NPAR_PAD = 5376;   // NPAR rounded up to 128 floats
constexpr size_t GRAD_SMEM = sizeof(float) * (NPAR_PAD + GRAD_R * 16 + 4 * GRAD_R * 64 + GRAD_R);

// One CTA takes a contiguous range of rows, 32 at a time: forward, backward,
// and the tile's gradient added to per-thread accumulators (thread t owns
// W2 entries t + 256q, W1 entries t + 256q and one bias or w3 entry).  The
// CTA's sums go to its own slot of `partial`, summed later in CTA order.
__global__ void __launch_bounds__(GRAD_T) k_merge_grad(const uint8_t *feat, const float *label, int64_t count,
                                                        const float *params, float *partial, double *loss_part) {
    extern __shared__ float sm[];
    float *sp = sm;
    float *sx = sp + NPAR_PAD;          // [R][16] scaled features
    float *sh1 = sx + GRAD_R * 16;      // [R][64]
    float *sh2 = sh1 + GRAD_R * 64;     // [R][64]
    float *sd2 = sh2 + GRAD_R * 64;     // [R][64] dL/dz2
    float *sd1 = sd2 + GRAD_R * 64;     // [R][64] dL/dz1
    float *sdo = sd1 + GRAD_R * 64;     // [R] dL/do
    __shared__ double s_loss[GRAD_T / 32];
    const int tid = threadIdx.x;
    for (int i = tid; i < NPAR; i += GRAD_T) sp[i] = params[i];
    const int64_t chunk = (count + gridDim.x - 1) / gridDim.x;
    const int64_t rb = (int64_t)blockIdx.x * chunk, re = min(count, rb + chunk);
    float gw2[16], gw1[4], gb = 0.f;
#pragma unroll
    for (int q = 0; q < 16; q++) gw2[q] = 0.f;
#pragma unroll
    for (int q = 0; q < 4; q++) gw1[q] = 0.f;
    double loss = 0.0;
    const float inv_count = count > 0 ? 1.0f / (float)count : 0.f;
    __syncthreads();
    for (int64_t r0 = rb; r0 < re; r0 += GRAD_R) {
        const int nr = (int)(re - r0 < GRAD_R ? re - r0 : GRAD_R);
        for (int t = tid; t < GRAD_R * 16; t += GRAD_T) {
            const int r = t >> 4;
            sx[t] = r < nr ? (float)feat[(r0 + r) * 16 + (t & 15)] * (1.0f / 256.0f) : 0.f;
        }
        __syncthreads();
        for (int t = tid; t < GRAD_R * 64; t += GRAD_T) {
            const int r = t >> 6, j = t & 63;
            float z = sp[P_B1 + j];
#pragma unroll
            for (int i = 0; i < 16; i++) z = fmaf(sp[P_W1 + j * 16 + i], sx[r * 16 + i], z);
            sh1[t] = fmaxf(z, 0.f);
        }
        __syncthreads();
        for (int t = tid; t < GRAD_R * 64; t += GRAD_T) {
            const int r = t >> 6, k = t & 63;
            float z = sp[P_B2 + k];
            for (int j = 0; j < 64; j++) z = fmaf(sp[P_W2 + k * 64 + j], sh1[r * 64 + j], z);
            sh2[t] = fmaxf(z, 0.f);
        }
        __syncthreads();
        if (tid < GRAD_R) {
            float d = 0.f;
            if (tid < nr) {
                float o = sp[P_B3];
                for (int k = 0; k < 64; k++) o = fmaf(sp[P_W3 + k], sh2[tid * 64 + k], o);
                const float y = label[r0 + tid];
                // stable binary cross-entropy of sigmoid(o): max(o,0) - o y + log(1 + e^-|o|)
                loss += (double)(fmaxf(o, 0.f) - o * y + log1pf(expf(-fabsf(o))));
                const float p = 1.0f / (1.0f + expf(-o));
                d = (p - y) * inv_count;
            }
            sdo[tid] = d;
        }
        __syncthreads();
        for (int t = tid; t < GRAD_R * 64; t += GRAD_T) {
            const int r = t >> 6, k = t & 63;
            sd2[t] = sh2[t] > 0.f ? sdo[r] * sp[P_W3 + k] : 0.f;
        }
        __syncthreads();
        for (int t = tid; t < GRAD_R * 64; t += GRAD_T) {
            const int r = t >> 6, j = t & 63;
            float a = 0.f;
            for (int k = 0; k < 64; k++) a = fmaf(sd2[r * 64 + k], sp[P_W2 + k * 64 + j], a);
            sd1[t] = sh1[t] > 0.f ? a : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 16; q++) {
            const int idx = tid + GRAD_T * q, k = idx >> 6, j = idx & 63;
            float a = gw2[q];
            for (int r = 0; r < GRAD_R; r++) a = fmaf(sd2[r * 64 + k], sh1[r * 64 + j], a);
            gw2[q] = a;
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int idx = tid + GRAD_T * q, j = idx >> 4, i = idx & 15;
            float a = gw1[q];
            for (int r = 0; r < GRAD_R; r++) a = fmaf(sd1[r * 64 + j], sx[r * 16 + i], a);
            gw1[q] = a;
        }
        if (tid < 64) {
            for (int r = 0; r < GRAD_R; r++) gb += sd1[r * 64 + tid];
        } else if (tid < 128) {
            for (int r = 0; r < GRAD_R; r++) gb += sd2[r * 64 + tid - 64];
        } else if (tid < 192) {
            for (int r = 0; r < GRAD_R; r++) gb = fmaf(sdo[r], sh2[r * 64 + tid - 128], gb);
        } else if (tid == 192) {
            for (int r = 0; r < GRAD_R; r++) gb += sdo[r];
        }
        __syncthreads();
    }
    float *pp = partial + (int64_t)blockIdx.x * NPAR;
#pragma unroll
    for (int q = 0; q < 16; q++) pp[P_W2 + tid + GRAD_T * q] = gw2[q];
#pragma unroll
    for (int q = 0; q < 4; q++) pp[P_W1 + tid + GRAD_T * q] = gw1[q];
    if (tid < 64) pp[P_B1 + tid] = gb;
    else if (tid < 128) pp[P_B2 + tid - 64] = gb;
    else if (tid < 192) pp[P_W3 + tid - 128] = gb;
    else if (tid == 192) pp[P_B3] = gb;
    // the loss terms live in the first warp
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_down_sync(0xffffffffu, loss, o);
    if ((tid & 31) == 0) s_loss[tid >> 5] = loss;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < GRAD_T / 32; w++) t += s_loss[w];
        loss_part[blockIdx.x] = t;
    }
}

// the CTAs' partial gradients summed in CTA order (deterministic)
__global__ void k_merge_grad_sum(const float *partial, const double *loss_part, int64_t count, float *grad,
                                 double *loss) {
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
    prepare_kernel((const void *)k_merge_grad, GRAD_T, GRAD_SMEM);
    k_merge_grad<<<GRAD_CTAS, GRAD_T, GRAD_SMEM, s>>>(feat, label, count, params, partial, lp);
    HP_LAUNCH_CHECK();
    k_merge_grad_sum<<<(NPAR + 255) / 256, 256, 0, s>>>(partial, lp, count, grad, lp + GRAD_CTAS);
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
    k_merge_adam<<<(NPAR + 255) / 256, 256, 0, s>>>(p, g, m, v, lr, b1, b2, eps, wd, c1, c2);
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
    k_merge_feats<<<grid_for((int64_t)X.n * X.K, 256), 256, 0, s>>>(Y);
    HP_LAUNCH_CHECK();
}

void merge_scores(const uint8_t *feat, int64_t count, const hp_merge_model *dmodel, int32_t *out, cudaStream_t s) {
    if (count <= 0) return;
    const int64_t tiles = cdiv(count, 16);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(tiles, MLP_WARPS), (int64_t)num_sms() * 8));
    k_merge_mlp<<<grid, MLP_WARPS * 32, 0, s>>>(feat, count, dmodel, out);
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
        k_merge_feats<<<grid_for(pairs, 256), 256, 0, s>>>(X);
        HP_LAUNCH_CHECK();
        merge_scores(X.feat, pairs, X.model, X.score, s);
        k_merge_select<<<grid_for(X.v1 - X.v0, 128), 128, 0, s>>>(X);
        HP_LAUNCH_CHECK();
    }
}

}  // namespace hp
