/*
 * hp_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU statement of the constrained multilevel
 * hypergraph partitioner of Ronzani & Silvano, "Hypergraph Partitioning on GPU
 * with Distinct Incident Hyperedges and Size Constraints".  It exists so that
 * the CUDA library can be checked against it, bit for bit.  Only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark load it;
 * the product path never does.  It shares no code, header or table with the
 * CUDA library.
 *
 * The method is a heuristic, so this file follows the paper's steps in the
 * paper's order and notation, one function per step:
 *   Sec. II     problem model, constraints, connectivity (Eq. 1)
 *   Sec. III    multilevel scheme, stop rule, projection of rho
 *   Sec. V-C    candidate pairs proposal: eta (Eq. 5), inter, valid (Eq. 6),
 *               deterministic symmetric noise, best-effort pairing of nodes
 *               left without a valid neighbour
 *   Sec. V-D    maximum-weight matching on the proposal pseudo-forest,
 *               Eq. 7-12, repeated for Pi proposal graphs
 *   Sec. V-E    coarse hypergraph construction (gamma, src/dst rule)
 *   Sec. VI-B   move proposal by gain (Eq. 13), size filter in the 2nd half
 *   Sec. VI-C   move chaining and sequence order, in-sequence gain (Eq. 14-15)
 *   Sec. VI-D   validity of every prefix, best valid prefix
 *
 * Readings where the paper is silent or ambiguous (each is part of the
 * contract the CUDA path must reproduce):
 *   - eta is fixed point: q(e) = floor(w(e) * 2^24 / |e|) (uint64).
 *   - noise(n,m) = SplitMix64-finaliser hash of (seed, level, min, max)
 *     reduced mod (cap+1); cap = floor(floor(sum_e q(e) / |E|) * permille/1000).
 *   - target ties go to the larger id (the max_id of Eq. 6).
 *   - round r of the matching targets the first still-unmatched entry of the
 *     node's top-Pi candidate list; a node without one is a tree root with
 *     ss1 = -inf; partner roots are excluded from child sets; a root that
 *     does not take its partner takes its best child only when ss1-0 > 0.
 *   - nodes with no valid neighbour are sorted by (size, id) and paired
 *     first-with-last when size and summed inbound counts fit.
 *   - coarse node id = rank of the cluster's smallest member; coarse
 *     hyperedges keep their id and weight, are never merged, singletons stay.
 *   - only moves with gain > 0 are proposed; ties of the move go to the
 *     larger partition id; moves sort by (p_s asc, gain desc, node asc).
 *   - chaining grade G = gain*10^7 - 10*|dsize| - |d|in|| (10^7 x the
 *     paper's grade with alpha = 1e-6, beta = 1e-7), chooser ties to the
 *     earlier sorted position, acceptor ties to the larger node id; chains
 *     ordered by (total gain desc, head node id asc), cycles start at their
 *     smallest node id.
 *   - Eq. 14-15 read additively: the in-sequence gain of a move is the exact
 *     change of connectivity it causes after all earlier moves.
 *   - best prefix: maximum cumulative gain over prefixes with zero violated
 *     partitions, ties to the longest; applied only when > 0.
 *   - a repetition that applies nothing ends its half of the repetitions
 *     (the next repetition would recompute the same moves).
 *   - count_kind = incident: every pin counts as a destination for the
 *     constraint (src sets emptied); the objective is unchanged.
 *
 * Learned merge priority (option learned_k; a growth of Sec. V-C that the
 * paper does not have): the top-K candidate lists by (eta, id), pairs kept
 * only when mutual, C(n) = top Pi of those by (s, eta, id) with s an integer
 * MLP 16 -> 64 -> 64 -> 1 of symmetric pair features; the matching weight
 * stays eta and the best-effort pairing still takes the nodes with no valid
 * neighbour.  Mutual lists keep the proposal graph free of cycles longer
 * than two.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

enum { OR_OK = 0, OR_ERR_INVALID_ARG = 1, OR_ERR_BAD_CSR = 2, OR_ERR_INFEASIBLE = 3 };

/* option vector layout shared with the Python wrapper of this file */
enum { OPT_PI, OPT_THETA, OPT_WINDOW, OPT_ROUNDS, OPT_PERMILLE, OPT_KIND, OPT_MAXLEV, OPT_LK, OPT_LL, OPT_N };
/* stats vector layout */
enum { ST_CONN, ST_CUTNET, ST_PARTS, ST_MAXSIZE, ST_MAXDIST, ST_VIOL, ST_LEVELS, ST_MOVES, ST_N = 16 };
/* per-level trace record layout */
/* per-level trace record layout; the last five describe the level's pairing:
 * nodes with a valid neighbour, nodes left without one (the best-effort
 * pairing's list), distinct targets and largest in-degree of the first
 * proposal graph, pairs of the first matching round */
enum { TR_N, TR_PINS, TR_PAIRS, TR_ISOPAIRS, TR_CONN, TR_MOVES, TR_REPS, TR_PARTS, TR_VALID, TR_ISOLIST, TR_TGT1,
       TR_MAXIN1, TR_PAIRS1, TR_W };

static void *xcalloc(size_t n, size_t sz)
{
    void *p = calloc(n ? n : 1, sz ? sz : 1);
    if (!p) {
        fprintf(stderr, "hp_oracle: out of memory\n");
        abort();
    }
    return p;
}

/* ------------------------------------------------------------------------ */
/* Sec. II: a level's directed hypergraph                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t n, e;     /* |N|, |E| */
    int64_t np;       /* sum_e |e| */
    int64_t *off;     /* [e+1] hyperedge segments */
    int32_t *pin;     /* [np] each segment: src(e) first, then dst(e) */
    int32_t *nsrc;    /* [e] |src(e)| */
    int32_t *w;       /* [e] omega(e) */
    int32_t *size;    /* [n] size(n) */
    int64_t *ioff;    /* [n+1] incidence segments */
    int32_t *inc;     /* in(n) ascending, then out(n) ascending */
    int32_t *nin;     /* [n] |in(n)| */
} hg_t;

static void hg_free(hg_t *g)
{
    free(g->off); free(g->pin); free(g->nsrc); free(g->w); free(g->size);
    free(g->ioff); free(g->inc); free(g->nin);
    memset(g, 0, sizeof *g);
}

static int64_t esize(const hg_t *g, int32_t e) { return g->off[e + 1] - g->off[e]; }
static int is_dst_pos(const hg_t *g, int32_t e, int64_t j) { return j - g->off[e] >= g->nsrc[e]; }

/* in(n) = {e : n in dst(e)}, out(n) = {e : n in src(e)} (Sec. II-A) */
static void hg_incidence(hg_t *g)
{
    int64_t *cnt = xcalloc((size_t)g->n + 1, sizeof(int64_t));
    int64_t *pin_pos = xcalloc((size_t)g->n + 1, sizeof(int64_t));
    int64_t *pout_pos = xcalloc((size_t)g->n + 1, sizeof(int64_t));
    g->nin = xcalloc((size_t)g->n, sizeof(int32_t));
    for (int32_t e = 0; e < g->e; e++)
        for (int64_t j = g->off[e]; j < g->off[e + 1]; j++) {
            cnt[g->pin[j] + 1]++;
            if (is_dst_pos(g, e, j)) g->nin[g->pin[j]]++;
        }
    g->ioff = xcalloc((size_t)g->n + 1, sizeof(int64_t));
    for (int32_t v = 0; v < g->n; v++) g->ioff[v + 1] = g->ioff[v] + cnt[v + 1];
    g->inc = xcalloc((size_t)g->np, sizeof(int32_t));
    for (int32_t v = 0; v < g->n; v++) {
        pin_pos[v] = g->ioff[v];
        pout_pos[v] = g->ioff[v] + g->nin[v];
    }
    for (int32_t e = 0; e < g->e; e++)
        for (int64_t j = g->off[e]; j < g->off[e + 1]; j++) {
            int32_t v = g->pin[j];
            if (is_dst_pos(g, e, j)) g->inc[pin_pos[v]++] = e;
            else g->inc[pout_pos[v]++] = e;
        }
    free(cnt); free(pin_pos); free(pout_pos);
}

/* ------------------------------------------------------------------------ */
/* Sec. V-C: histogram over neighbours, Eq. 5, with fixed-point weights       */
/* ------------------------------------------------------------------------ */
static uint64_t splitmix64_mix(uint64_t z)
{
    /* finaliser of SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) */
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* symmetric deterministic noise rng(min(n,m), max(n,m)) capped at cap */
static uint64_t pair_noise(uint64_t seed, int32_t level, int32_t a, int32_t b, uint64_t cap)
{
    uint32_t lo = (uint32_t)(a < b ? a : b), hi = (uint32_t)(a < b ? b : a);
    uint64_t h = splitmix64_mix(seed + 0x9E3779B97F4A7C15ULL * (uint64_t)(level + 1));
    h = splitmix64_mix(h ^ (((uint64_t)lo << 32) | (uint64_t)hi));
    return h % (cap + 1);
}

/* q(e) = floor(omega(e) * 2^24 / |e|); returns the noise cap of the level */
static uint64_t level_weights(const hg_t *g, uint64_t *q, int32_t permille)
{
    uint64_t sum = 0;
    for (int32_t e = 0; e < g->e; e++) {
        q[e] = ((uint64_t)g->w[e] << 24) / (uint64_t)esize(g, e);
        sum += q[e];
    }
    if (g->e == 0) return 0;
    return (sum / (uint64_t)g->e) * (uint64_t)permille / 1000u;
}

/* For node v: eta0[m] = sum_{e in I(v), m in e} q(e) (Eq. 5 without noise),
 * inter[m] = |in(v) intersect in(m)|, for every m in N(v) (listed in nb). */
static int32_t node_histogram(const hg_t *g, const uint64_t *q, int32_t v, uint64_t *eta0,
                              int32_t *inter, uint8_t *seen, int32_t *nb)
{
    int32_t k = 0;
    for (int64_t t = g->ioff[v]; t < g->ioff[v + 1]; t++) {
        int32_t e = g->inc[t];
        int v_inbound = t < g->ioff[v] + g->nin[v];
        for (int64_t j = g->off[e]; j < g->off[e + 1]; j++) {
            int32_t m = g->pin[j];
            if (m == v) continue;
            if (!seen[m]) {
                seen[m] = 1;
                nb[k++] = m;
            }
            eta0[m] += q[e];
            if (v_inbound && is_dst_pos(g, e, j)) inter[m]++;
        }
    }
    return k;
}

/* valid(n, m) of Eq. 6, with |in(n) U in(m)| = |in(n)| + |in(m)| - inter */
static int pair_valid(const hg_t *g, int32_t v, int32_t m, int32_t inter, int32_t omega, int32_t delta)
{
    if ((int64_t)g->size[v] + g->size[m] > omega) return 0;
    return (int64_t)g->nin[v] + g->nin[m] - inter <= delta;
}

static int key_gt(uint64_t e1, int32_t m1, uint64_t e2, int32_t m2)
{
    return e1 > e2 || (e1 == e2 && m1 > m2);
}

/* top-Pi valid neighbours of every node, by (eta, id) descending (Eq. 6) */
static void propose_pairs(const hg_t *g, int32_t level, uint64_t seed, int32_t omega, int32_t delta,
                          int32_t pi, int32_t permille, int32_t *cand, uint64_t *cscore)
{
    uint64_t *q = xcalloc((size_t)g->e, sizeof(uint64_t));
    uint64_t cap = level_weights(g, q, permille);
    uint64_t *eta0 = xcalloc((size_t)g->n, sizeof(uint64_t));
    int32_t *inter = xcalloc((size_t)g->n, sizeof(int32_t));
    uint8_t *seen = xcalloc((size_t)g->n, 1);
    int32_t *nb = xcalloc((size_t)g->n, sizeof(int32_t));
    for (int32_t v = 0; v < g->n; v++) {
        int32_t k = node_histogram(g, q, v, eta0, inter, seen, nb);
        int32_t *cv = cand + (int64_t)v * pi;
        uint64_t *sv = cscore + (int64_t)v * pi;
        int32_t have = 0;
        for (int32_t i = 0; i < pi; i++) { cv[i] = -1; sv[i] = 0; }
        for (int32_t i = 0; i < k; i++) {
            int32_t m = nb[i];
            if (pair_valid(g, v, m, inter[m], omega, delta)) {
                uint64_t eta = eta0[m] + pair_noise(seed, level, v, m, cap);
                /* insert into the sorted top-Pi list */
                int32_t pos = have;
                while (pos > 0 && key_gt(eta, m, sv[pos - 1], cv[pos - 1])) pos--;
                if (pos < pi) {
                    int32_t last = have < pi ? have : pi - 1;
                    for (int32_t s = last; s > pos; s--) { cv[s] = cv[s - 1]; sv[s] = sv[s - 1]; }
                    cv[pos] = m;
                    sv[pos] = eta;
                    if (have < pi) have++;
                }
            }
            eta0[m] = 0;
            inter[m] = 0;
            seen[m] = 0;
        }
    }
    free(q); free(eta0); free(inter); free(seen); free(nb);
}

/* ------------------------------------------------------------------------ */
/* Sec. V-C: best-effort pairing of nodes left without a valid neighbour      */
/* ------------------------------------------------------------------------ */
typedef struct { int32_t size, id; } sz_id_t;

static int cmp_sz_id(const void *a, const void *b)
{
    const sz_id_t *x = a, *y = b;
    if (x->size != y->size) return x->size < y->size ? -1 : 1;
    return x->id < y->id ? -1 : (x->id > y->id);
}

static int64_t pair_isolated(const hg_t *g, int32_t pi, const int32_t *cand, int32_t omega,
                             int32_t delta, int32_t *mate)
{
    sz_id_t *L = xcalloc((size_t)g->n, sizeof(sz_id_t));
    int32_t k = 0;
    for (int32_t v = 0; v < g->n; v++)
        if (mate[v] < 0 && cand[(int64_t)v * pi] < 0) { L[k].size = g->size[v]; L[k].id = v; k++; }
    qsort(L, (size_t)k, sizeof(sz_id_t), cmp_sz_id);
    int64_t pairs = 0;
    for (int32_t i = 0; i < k / 2; i++) {
        int32_t a = L[i].id, b = L[k - 1 - i].id;
        /* the inbound union is over-estimated by the sum of inbound counts */
        if ((int64_t)g->size[a] + g->size[b] <= omega && (int64_t)g->nin[a] + g->nin[b] <= delta) {
            mate[a] = b;
            mate[b] = a;
            pairs++;
        }
    }
    free(L);
    return pairs;
}

/* ------------------------------------------------------------------------ */
/* Sec. V-D: maximum-weight matching on one proposal graph (Eq. 7-12)         */
/* ------------------------------------------------------------------------ */
/* target[v] = -1 when undefined.  Writes mate[] for the pairs it forms and
 * returns their number.  R = nodes on 2-cycles; child(n) excludes R. */
static int64_t match_round(int32_t n, const int32_t *target, const uint64_t *score, int32_t *mate)
{
    uint8_t *inR = xcalloc((size_t)n, 1);
    int64_t *coff = xcalloc((size_t)n + 1, sizeof(int64_t));
    int32_t *kids = xcalloc((size_t)n, sizeof(int32_t));
    int64_t *fill = xcalloc((size_t)n, sizeof(int64_t));
    int64_t *ss0 = xcalloc((size_t)n, sizeof(int64_t));
    int64_t *ss1 = xcalloc((size_t)n, sizeof(int64_t));
    int64_t *sum0 = xcalloc((size_t)n, sizeof(int64_t));
    int32_t *best = xcalloc((size_t)n, sizeof(int32_t));
    uint8_t *up = xcalloc((size_t)n, 1);
    int32_t *stack = xcalloc((size_t)n + 1, sizeof(int32_t));
    int32_t *order = xcalloc((size_t)n + 1, sizeof(int32_t));

    for (int32_t v = 0; v < n; v++) {
        int32_t t = target[v];
        inR[v] = t >= 0 && target[t] == v;
    }
    /* child(n) \ R as CSR, children in ascending id */
    for (int32_t v = 0; v < n; v++)
        if (target[v] >= 0 && !inR[v]) coff[target[v] + 1]++;
    for (int32_t v = 0; v < n; v++) coff[v + 1] += coff[v];
    for (int32_t v = 0; v < n; v++) fill[v] = coff[v];
    for (int32_t v = 0; v < n; v++)
        if (target[v] >= 0 && !inR[v]) kids[fill[target[v]]++] = v;

    /* bottom-up: a pre-order from every root, then read backwards */
    int32_t no = 0;
    for (int32_t r = 0; r < n; r++) {
        if (!(target[r] < 0 || inR[r])) continue;
        int32_t sp = 0;
        stack[sp++] = r;
        while (sp) {
            int32_t v = stack[--sp];
            order[no++] = v;
            for (int64_t c = coff[v]; c < coff[v + 1]; c++) stack[sp++] = kids[c];
        }
    }
    for (int32_t i = no - 1; i >= 0; i--) {
        int32_t v = order[i];
        int64_t s0 = 0;
        int32_t b = -1;
        for (int64_t c = coff[v]; c < coff[v + 1]; c++) {
            int32_t k = kids[c];
            s0 += ss0[k];
            /* argmax over children of (ss1-0, id) */
            if (b < 0 || ss1[k] - ss0[k] > ss1[b] - ss0[b] ||
                (ss1[k] - ss0[k] == ss1[b] - ss0[b] && k > b))
                b = k;
        }
        sum0[v] = s0;
        best[v] = b;
        /* Eq. 10 */
        ss0[v] = s0 + ((b >= 0 && ss1[b] - ss0[b] > 0) ? ss1[b] - ss0[b] : 0);
        /* Eq. 7 (non-roots); roots are completed below */
        if (target[v] >= 0 && !inR[v]) ss1[v] = (int64_t)score[v] + s0;
    }
    /* Eq. 8 for roots on a 2-cycle; Eq. 11 decides them */
    for (int32_t v = 0; v < n; v++)
        if (inR[v]) ss1[v] = (int64_t)score[v] + sum0[v] + sum0[target[v]];
    for (int32_t v = 0; v < n; v++)
        if (inR[v]) up[v] = ss1[v] > ss0[v] + ss0[target[v]];
    /* top-down, Eq. 12: the order array is a pre-order, parents first */
    for (int32_t i = 0; i < no; i++) {
        int32_t v = order[i];
        if (target[v] >= 0 && !inR[v]) {
            int32_t t = target[v];
            up[v] = !up[t] && best[t] == v && ss1[v] - ss0[v] > 0;
        }
    }
    int64_t pairs = 0;
    for (int32_t v = 0; v < n; v++)
        if (up[v]) {
            mate[v] = target[v];
            mate[target[v]] = v;
            if (v < target[v] || !inR[v]) pairs++;
        }
    free(inR); free(coff); free(kids); free(fill); free(ss0); free(ss1); free(sum0);
    free(best); free(up); free(stack); free(order);
    return pairs;
}

/* Pi rounds; nodes matched earlier leave later proposal graphs (Sec. V-D).
 * r1 (NULL or 3 values): distinct targets and largest in-degree of the first
 * proposal graph, pairs formed by the first round. */
static int64_t match_all(int32_t n, int32_t pi, const int32_t *cand, const uint64_t *cscore, int32_t *mate,
                         int64_t *r1)
{
    int32_t *target = xcalloc((size_t)n, sizeof(int32_t));
    uint64_t *score = xcalloc((size_t)n, sizeof(uint64_t));
    int32_t *rmate = xcalloc((size_t)n, sizeof(int32_t));
    int64_t pairs = 0;
    for (int32_t r = 0; r < pi; r++) {
        for (int32_t v = 0; v < n; v++) {
            target[v] = -1;
            score[v] = 0;
            rmate[v] = -1;
            if (mate[v] >= 0) continue;
            for (int32_t i = 0; i < pi; i++) {
                int32_t c = cand[(int64_t)v * pi + i];
                if (c < 0) break;
                if (mate[c] < 0) {
                    target[v] = c;
                    score[v] = cscore[(int64_t)v * pi + i];
                    break;
                }
            }
        }
        if (r == 0 && r1) {
            int32_t *indeg = xcalloc((size_t)n + 1, sizeof(int32_t));
            for (int32_t v = 0; v < n; v++)
                if (target[v] >= 0) indeg[target[v]]++;
            r1[0] = r1[1] = 0;
            for (int32_t v = 0; v < n; v++) {
                if (indeg[v] > 0) r1[0]++;
                if (indeg[v] > r1[1]) r1[1] = indeg[v];
            }
            free(indeg);
        }
        int64_t pr = match_round(n, target, score, rmate);
        if (r == 0 && r1) r1[2] = pr;
        pairs += pr;
        for (int32_t v = 0; v < n; v++)
            if (rmate[v] >= 0) mate[v] = rmate[v];
    }
    free(target); free(score); free(rmate);
    return pairs;
}

/* ------------------------------------------------------------------------ */
/* Learned merge priority: a growth of Sec. V-C that is not in the paper.      */
/* Each node keeps its top-K valid candidates by (eta, id) (Eq. 6 with K for  */
/* Pi); a pair is kept only when each end is in the other's list, and C(n) is  */
/* the top Pi of those by (s, eta, id), s being an integer MLP of sixteen      */
/* symmetric pair features.  The matching weight stays eta.                   */
/* ------------------------------------------------------------------------ */
enum { ML_IN = 16, ML_HID = 64 };
/* model vector layout shared with the Python wrapper of this file */
enum {
    MD_W1 = 0,                          /* [64][16] codes in [-127, 127] */
    MD_W2 = MD_W1 + ML_HID * ML_IN,     /* [64][64] */
    MD_W3 = MD_W2 + ML_HID * ML_HID,    /* [64] */
    MD_B1 = MD_W3 + ML_HID,             /* [64], |b| <= 2^30 */
    MD_B2 = MD_B1 + ML_HID,             /* [64] */
    MD_B3 = MD_B2 + ML_HID,
    MD_S1, MD_S2,                       /* right shifts, 0..30 */
    MD_N
};

static int model_ok(const int32_t *md)
{
    for (int i = MD_W1; i < MD_B1; i++)
        if (md[i] < -127 || md[i] > 127) return 0;
    for (int i = MD_B1; i <= MD_B3; i++)
        if (md[i] < -(1 << 30) || md[i] > (1 << 30)) return 0;
    return md[MD_S1] >= 0 && md[MD_S1] <= 30 && md[MD_S2] >= 0 && md[MD_S2] <= 30;
}

/* log code of x >= 0: 0 for 0, else 1 + 4 floor(log2 x) + the two bits after
 * the leading one, at most 255 */
static int32_t log_code(uint64_t x)
{
    if (x == 0) return 0;
    int b = 63;
    while (!((x >> b) & 1u)) b--;
    uint64_t frac = b >= 2 ? (x >> (b - 2)) & 3u : (x << (2 - b)) & 3u;
    int64_t c = 1 + 4 * (int64_t)b + (int64_t)frac;
    return (int32_t)(c > 255 ? 255 : c);
}

static int32_t imin32(int32_t a, int32_t b) { return a < b ? a : b; }
static int32_t imax32(int32_t a, int32_t b) { return a > b ? a : b; }

/* The sixteen features of the pair (v, m), each in 0..255 and each symmetric
 * in v and m.  eta is the pair's Eq. 5 value with noise; rv, rm the
 * positions of m in v's list and of v in m's list.  emark is a zeroed
 * scratch of |E| bytes, left zeroed. */
static void pair_features(const hg_t *g, int32_t level, int32_t v, int32_t m, uint64_t eta, int32_t rv,
                          int32_t rm, int32_t omega, int32_t delta, uint8_t *emark, uint8_t *f)
{
    /* hyperedges holding both ends (shared) and inbound to both (inter) */
    for (int64_t t = g->ioff[m]; t < g->ioff[m + 1]; t++)
        emark[g->inc[t]] = t < g->ioff[m] + g->nin[m] ? 1 : 2;
    int64_t shared = 0, inter = 0;
    for (int64_t t = g->ioff[v]; t < g->ioff[v + 1]; t++) {
        uint8_t k = emark[g->inc[t]];
        if (k) shared++;
        if (k == 1 && t < g->ioff[v] + g->nin[v]) inter++;
    }
    for (int64_t t = g->ioff[m]; t < g->ioff[m + 1]; t++) emark[g->inc[t]] = 0;
    int64_t sv = g->size[v], sm = g->size[m], iv = g->nin[v], im = g->nin[m];
    int64_t dv = g->ioff[v + 1] - g->ioff[v], dm = g->ioff[m + 1] - g->ioff[m];
    int64_t uni = iv + im - inter;
    f[0] = (uint8_t)log_code(eta);
    f[1] = (uint8_t)log_code((uint64_t)shared);
    f[2] = (uint8_t)log_code((uint64_t)inter);
    f[3] = (uint8_t)log_code((uint64_t)(sv < sm ? sv : sm));
    f[4] = (uint8_t)log_code((uint64_t)(sv > sm ? sv : sm));
    f[5] = (uint8_t)log_code((uint64_t)(iv < im ? iv : im));
    f[6] = (uint8_t)log_code((uint64_t)(iv > im ? iv : im));
    f[7] = (uint8_t)log_code((uint64_t)(dv < dm ? dv : dm));
    f[8] = (uint8_t)log_code((uint64_t)(dv > dm ? dv : dm));
    f[9] = (uint8_t)(255 * (sv + sm) / omega);              /* valid: sv + sm <= omega */
    f[10] = (uint8_t)(delta > 0 ? 255 * uni / delta : 0);   /* valid: uni <= delta */
    f[11] = (uint8_t)(level < 255 ? level : 255);
    f[12] = (uint8_t)(uni > 0 ? 255 * inter / uni : 0);
    f[13] = (uint8_t)imin32(rv, rm);
    f[14] = (uint8_t)imax32(rv, rm);
    f[15] = (uint8_t)log_code((uint64_t)(iv + im));
}

/* s = b3 + w3 . a2, a2 = clamp((b2 + W2 a1) >> s2, 0, 255),
 * a1 = clamp((b1 + W1 f) >> s1, 0, 255): integers throughout */
static int64_t mlp_score(const int32_t *md, const uint8_t *f)
{
    int64_t a1[ML_HID], a2[ML_HID];
    for (int j = 0; j < ML_HID; j++) {
        int64_t h = md[MD_B1 + j];
        for (int i = 0; i < ML_IN; i++) h += (int64_t)md[MD_W1 + j * ML_IN + i] * f[i];
        a1[j] = h <= 0 ? 0 : ((h >> md[MD_S1]) > 255 ? 255 : (h >> md[MD_S1]));
    }
    for (int k = 0; k < ML_HID; k++) {
        int64_t h = md[MD_B2 + k];
        for (int j = 0; j < ML_HID; j++) h += (int64_t)md[MD_W2 + k * ML_HID + j] * a1[j];
        a2[k] = h <= 0 ? 0 : ((h >> md[MD_S2]) > 255 ? 255 : (h >> md[MD_S2]));
    }
    int64_t out = md[MD_B3];
    for (int k = 0; k < ML_HID; k++) out += (int64_t)md[MD_W3 + k] * a2[k];
    return out;
}

static int learned_gt(int64_t s1, uint64_t e1, int32_t m1, int64_t s2, uint64_t e2, int32_t m2)
{
    if (s1 != s2) return s1 > s2;
    return key_gt(e1, m1, e2, m2);
}

/* C(n) of the learned priority from the top-K lists candK/csK */
static void learned_candidates(const hg_t *g, int32_t level, int32_t K, const int32_t *candK, const uint64_t *csK,
                               int32_t pi, const int32_t *md, int32_t omega, int32_t delta, int32_t *cand,
                               uint64_t *cscore)
{
    uint8_t *emark = xcalloc((size_t)g->e + 1, 1);
    int64_t *sk = xcalloc((size_t)pi, sizeof(int64_t));
    for (int32_t v = 0; v < g->n; v++) {
        int32_t *cv = cand + (int64_t)v * pi;
        uint64_t *ev = cscore + (int64_t)v * pi;
        int32_t have = 0;
        for (int32_t i = 0; i < pi; i++) { cv[i] = -1; ev[i] = 0; }
        for (int32_t j = 0; j < K; j++) {
            int32_t m = candK[(int64_t)v * K + j];
            if (m < 0) break;
            int32_t rm = -1;
            for (int32_t i = 0; i < K; i++)
                if (candK[(int64_t)m * K + i] == v) { rm = i; break; }
            if (rm < 0) continue;   /* v is not among m's candidates */
            uint8_t f[ML_IN];
            uint64_t eta = csK[(int64_t)v * K + j];
            pair_features(g, level, v, m, eta, j, rm, omega, delta, emark, f);
            int64_t s = mlp_score(md, f);
            int32_t pos = have;
            while (pos > 0 && learned_gt(s, eta, m, sk[pos - 1], ev[pos - 1], cv[pos - 1])) pos--;
            if (pos < pi) {
                int32_t last = have < pi ? have : pi - 1;
                for (int32_t t = last; t > pos; t--) { cv[t] = cv[t - 1]; ev[t] = ev[t - 1]; sk[t] = sk[t - 1]; }
                cv[pos] = m;
                ev[pos] = eta;
                sk[pos] = s;
                if (have < pi) have++;
            }
        }
    }
    free(emark);
    free(sk);
}

/* ------------------------------------------------------------------------ */
/* Sec. V-E: coarse hypergraph                                               */
/* ------------------------------------------------------------------------ */
static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return x < y ? -1 : (x > y);
}

static int32_t sort_unique(int32_t *a, int32_t k)
{
    qsort(a, (size_t)k, sizeof(int32_t), cmp_i32);
    int32_t u = 0;
    for (int32_t i = 0; i < k; i++)
        if (u == 0 || a[i] != a[u - 1]) a[u++] = a[i];
    return u;
}

static int contains_sorted(const int32_t *a, int32_t k, int32_t x)
{
    int32_t lo = 0, hi = k;
    while (lo < hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo < k && a[lo] == x;
}

/* gamma(n) = rank of min(n, match(n)); dst' = gamma(dst(e)),
 * src' = gamma(src(e)) \ dst'; omega' = omega. */
static void contract(const hg_t *g, const int32_t *mate, hg_t *c, int32_t *gamma)
{
    int32_t *rank = xcalloc((size_t)g->n, sizeof(int32_t));
    int32_t nc = 0;
    for (int32_t v = 0; v < g->n; v++)
        if (mate[v] < 0 || v < mate[v]) rank[v] = nc++;
    for (int32_t v = 0; v < g->n; v++) gamma[v] = rank[(mate[v] >= 0 && mate[v] < v) ? mate[v] : v];
    memset(c, 0, sizeof *c);
    c->n = nc;
    c->e = g->e;
    c->size = xcalloc((size_t)nc, sizeof(int32_t));
    for (int32_t v = 0; v < g->n; v++) c->size[gamma[v]] += g->size[v];
    c->w = xcalloc((size_t)g->e, sizeof(int32_t));
    memcpy(c->w, g->w, sizeof(int32_t) * (size_t)g->e);
    c->nsrc = xcalloc((size_t)g->e, sizeof(int32_t));
    c->off = xcalloc((size_t)g->e + 1, sizeof(int64_t));
    c->pin = xcalloc((size_t)g->np, sizeof(int32_t));
    int32_t *sbuf = xcalloc((size_t)g->np + 1, sizeof(int32_t));
    int32_t *dbuf = xcalloc((size_t)g->np + 1, sizeof(int32_t));
    int64_t at = 0;
    for (int32_t e = 0; e < g->e; e++) {
        int32_t ns = 0, nd = 0;
        for (int64_t j = g->off[e]; j < g->off[e + 1]; j++) {
            if (is_dst_pos(g, e, j)) dbuf[nd++] = gamma[g->pin[j]];
            else sbuf[ns++] = gamma[g->pin[j]];
        }
        nd = sort_unique(dbuf, nd);
        ns = sort_unique(sbuf, ns);
        int32_t ks = 0;
        for (int32_t i = 0; i < ns; i++)
            if (!contains_sorted(dbuf, nd, sbuf[i])) sbuf[ks++] = sbuf[i];
        c->off[e] = at;
        for (int32_t i = 0; i < ks; i++) c->pin[at++] = sbuf[i];
        for (int32_t i = 0; i < nd; i++) c->pin[at++] = dbuf[i];
        c->nsrc[e] = ks;
    }
    c->off[g->e] = at;
    c->np = at;
    free(sbuf); free(dbuf); free(rank);
    hg_incidence(c);
}

/* ------------------------------------------------------------------------ */
/* Sec. II-B: objective and constraint state of a partitioning                */
/* ------------------------------------------------------------------------ */
/* pins(p, e) as a short list per hyperedge: entries (p, pins, pins_in),
 * list of e at [2*off[e], 2*off[e] + len[e]); capacity 2|e| leaves room for
 * one destination partition per pin during sequence simulation. */
typedef struct {
    int32_t *p, *cnt, *cin, *len;
} plist_t;

static void plist_alloc(const hg_t *g, plist_t *L)
{
    L->p = xcalloc((size_t)(2 * g->np), sizeof(int32_t));
    L->cnt = xcalloc((size_t)(2 * g->np), sizeof(int32_t));
    L->cin = xcalloc((size_t)(2 * g->np), sizeof(int32_t));
    L->len = xcalloc((size_t)g->e, sizeof(int32_t));
}

static void plist_free(plist_t *L) { free(L->p); free(L->cnt); free(L->cin); free(L->len); }

static int64_t plist_find(const hg_t *g, const plist_t *L, int32_t e, int32_t p)
{
    int64_t base = 2 * g->off[e];
    for (int32_t i = 0; i < L->len[e]; i++)
        if (L->p[base + i] == p) return base + i;
    return -1;
}

static int64_t plist_find_or_add(const hg_t *g, plist_t *L, int32_t e, int32_t p)
{
    int64_t k = plist_find(g, L, e, p);
    if (k >= 0) return k;
    k = 2 * g->off[e] + L->len[e]++;
    L->p[k] = p;
    L->cnt[k] = 0;
    L->cin[k] = 0;
    return k;
}

/* pins(p,e), pins_in(p,e) for the current rho */
static void plist_build(const hg_t *g, const int32_t *rho, plist_t *L)
{
    for (int32_t e = 0; e < g->e; e++) {
        L->len[e] = 0;
        for (int64_t j = g->off[e]; j < g->off[e + 1]; j++) {
            int64_t k = plist_find_or_add(g, L, e, rho[g->pin[j]]);
            L->cnt[k]++;
            if (is_dst_pos(g, e, j)) L->cin[k]++;
        }
    }
}

/* Eq. 1 connectivity and Eq. 16 cut-net */
static void objective(const hg_t *g, const int32_t *rho, int32_t nparts, int64_t *conn, int64_t *cutnet)
{
    int32_t *mark = xcalloc((size_t)nparts, sizeof(int32_t));
    int64_t c = 0, cn = 0;
    for (int32_t e = 0; e < g->e; e++) {
        int64_t lambda = 0;
        for (int64_t j = g->off[e]; j < g->off[e + 1]; j++) {
            int32_t p = rho[g->pin[j]];
            if (mark[p] != e + 1) { mark[p] = e + 1; lambda++; }
        }
        c += (int64_t)g->w[e] * (lambda - 1);
        if (lambda > 1) cn += g->w[e];
    }
    free(mark);
    *conn = c;
    *cutnet = cn;
}

/* ------------------------------------------------------------------------ */
/* Sec. VI-B: moves proposed in isolation, Eq. 13                             */
/* ------------------------------------------------------------------------ */
typedef struct { int32_t node, src, dst; int64_t gain; } move_t;

static int32_t propose_moves(const hg_t *g, const int32_t *rho, int32_t nparts, const plist_t *L,
                             const int64_t *psize, int32_t omega, int second_half, move_t *mv)
{
    int64_t *conn = xcalloc((size_t)nparts, sizeof(int64_t));
    uint8_t *touched = xcalloc((size_t)nparts, 1);
    int32_t *tl = xcalloc((size_t)nparts, sizeof(int32_t));
    int32_t m = 0;
    for (int32_t v = 0; v < g->n; v++) {
        int32_t s = rho[v];
        int64_t W = 0, saving = 0;
        int32_t nt = 0;
        for (int64_t t = g->ioff[v]; t < g->ioff[v + 1]; t++) {
            int32_t e = g->inc[t];
            int64_t base = 2 * g->off[e];
            W += g->w[e];
            for (int32_t i = 0; i < L->len[e]; i++) {
                int32_t p = L->p[base + i];
                if (p == s) {
                    if (L->cnt[base + i] == 1) saving += g->w[e];
                } else {
                    if (!touched[p]) { touched[p] = 1; tl[nt++] = p; }
                    conn[p] += g->w[e];
                }
            }
        }
        /* gain(n,p) = saving(n) - loss(n,p), loss(n,p) = W(n) - conn(n,p) */
        int32_t bp = -1;
        int64_t bg = 0;
        for (int32_t i = 0; i < nt; i++) {
            int32_t p = tl[i];
            int ok = !second_half || (int64_t)g->size[v] + psize[p] <= omega;
            int64_t gain = saving - (W - conn[p]);
            if (ok && (bp < 0 || gain > bg || (gain == bg && p > bp))) { bp = p; bg = gain; }
            conn[p] = 0;
            touched[p] = 0;
        }
        if (bp >= 0 && bg > 0) {
            mv[m].node = v; mv[m].src = s; mv[m].dst = bp; mv[m].gain = bg;
            m++;
        }
    }
    free(conn); free(touched); free(tl);
    return m;
}

static int cmp_move(const void *a, const void *b)
{
    const move_t *x = a, *y = b;
    if (x->src != y->src) return x->src < y->src ? -1 : 1;
    if (x->gain != y->gain) return x->gain > y->gain ? -1 : 1;
    return x->node < y->node ? -1 : (x->node > y->node);
}

/* ------------------------------------------------------------------------ */
/* Sec. VI-C: chains of moves and the sequence order                          */
/* ------------------------------------------------------------------------ */
typedef struct { int64_t gain; int32_t head_node, first; } chain_t;

static int cmp_chain(const void *a, const void *b)
{
    const chain_t *x = a, *y = b;
    if (x->gain != y->gain) return x->gain > y->gain ? -1 : 1;
    return x->head_node < y->head_node ? -1 : (x->head_node > y->head_node);
}

static __int128 grade(const hg_t *g, const move_t *n, const move_t *m)
{
    int64_t ds = (int64_t)g->size[n->node] - g->size[m->node];
    int64_t di = (int64_t)g->nin[n->node] - g->nin[m->node];
    if (ds < 0) ds = -ds;
    if (di < 0) di = -di;
    return (__int128)m->gain * 10000000 - (__int128)10 * ds - di;
}

/* mv sorted; writes seq[k] = index into mv of the k-th move of the sequence */
static void sequence_moves(const hg_t *g, int32_t nparts, const move_t *mv, int32_t M, int32_t window,
                           int32_t rounds, int32_t *seq)
{
    int32_t *pred = xcalloc((size_t)M + 1, sizeof(int32_t));
    int32_t *succ = xcalloc((size_t)M + 1, sizeof(int32_t));
    int32_t *pred0 = xcalloc((size_t)M + 1, sizeof(int32_t));
    int32_t *choice = xcalloc((size_t)M + 1, sizeof(int32_t));
    __int128 *cg = xcalloc((size_t)M + 1, sizeof(__int128));
    int32_t *acc = xcalloc((size_t)M + 1, sizeof(int32_t));
    int64_t *first = xcalloc((size_t)nparts + 1, sizeof(int64_t));
    for (int32_t i = 0; i < M; i++) { pred[i] = -1; succ[i] = -1; }
    /* moves leaving partition p are the sorted range [first[p], first[p+1]) */
    for (int32_t i = 0; i < M; i++) first[mv[i].src + 1]++;
    for (int32_t p = 0; p < nparts; p++) first[p + 1] += first[p];

    for (int32_t t = 0; t < rounds; t++) {
        memcpy(pred0, pred, sizeof(int32_t) * (size_t)M);
        for (int32_t i = 0; i < M; i++) {
            choice[i] = -1;
            if (succ[i] >= 0) continue; /* only free chain ends choose */
            int32_t d = mv[i].dst;
            int32_t seen = 0;
            for (int64_t j = first[d]; j < first[d + 1] && seen < window; j++) {
                if (pred0[j] >= 0 || j == i) continue;
                seen++;
                __int128 G = grade(g, &mv[i], &mv[j]);
                if (choice[i] < 0 || G > cg[i]) { choice[i] = (int32_t)j; cg[i] = G; }
            }
        }
        /* conflicts: the chosen move takes the chooser of max (G, node id) */
        for (int32_t j = 0; j < M; j++) acc[j] = -1;
        for (int32_t i = 0; i < M; i++) {
            int32_t j = choice[i];
            if (j < 0) continue;
            int32_t a = acc[j];
            if (a < 0 || cg[i] > cg[a] || (cg[i] == cg[a] && mv[i].node > mv[a].node)) acc[j] = i;
        }
        int any = 0;
        for (int32_t j = 0; j < M; j++)
            if (acc[j] >= 0) {
                pred[j] = acc[j];
                succ[acc[j]] = j;
                any = 1;
            }
        if (!any) break;
    }
    /* chains: paths from their head, then cycles from their smallest node id */
    uint8_t *vis = xcalloc((size_t)M + 1, 1);
    chain_t *ch = xcalloc((size_t)M + 1, sizeof(chain_t));
    int32_t nch = 0;
    for (int32_t i = 0; i < M; i++) {
        if (pred[i] >= 0) continue;
        int64_t gsum = 0;
        for (int32_t j = i; j >= 0; j = succ[j]) { vis[j] = 1; gsum += mv[j].gain; }
        ch[nch].gain = gsum; ch[nch].head_node = mv[i].node; ch[nch].first = i;
        nch++;
    }
    for (int32_t i = 0; i < M; i++) {
        if (vis[i]) continue;
        int32_t h = i;
        int64_t gsum = 0;
        int32_t j = i;
        do {
            vis[j] = 1;
            gsum += mv[j].gain;
            if (mv[j].node < mv[h].node) h = j;
            j = succ[j];
        } while (j != i);
        ch[nch].gain = gsum; ch[nch].head_node = mv[h].node; ch[nch].first = h;
        nch++;
    }
    qsort(ch, (size_t)nch, sizeof(chain_t), cmp_chain);
    int32_t k = 0;
    for (int32_t c = 0; c < nch; c++) {
        int32_t j = ch[c].first;
        do {
            seq[k++] = j;
            j = succ[j];
        } while (j >= 0 && j != ch[c].first);
    }
    free(pred); free(succ); free(pred0); free(choice); free(cg); free(acc); free(first);
    free(vis); free(ch);
}

/* Eq. 14-15 (additive reading): gain of each move after all earlier moves */
static void inseq_gains(const hg_t *g, const int32_t *rho, const move_t *mv, const int32_t *seq,
                        int32_t M, int64_t *gseq)
{
    plist_t L;
    plist_alloc(g, &L);
    plist_build(g, rho, &L);
    for (int32_t k = 0; k < M; k++) {
        const move_t *x = &mv[seq[k]];
        int64_t gk = 0;
        for (int64_t t = g->ioff[x->node]; t < g->ioff[x->node + 1]; t++) {
            int32_t e = g->inc[t];
            int64_t ks = plist_find(g, &L, e, x->src);
            int64_t kd = plist_find_or_add(g, &L, e, x->dst);
            if (L.cnt[ks] == 1) gk += g->w[e]; /* n is the last pin of e leaving p_s */
            if (L.cnt[kd] == 0) gk -= g->w[e]; /* n is the first pin of e entering p_d */
            L.cnt[ks]--;
            L.cnt[kd]++;
        }
        gseq[k] = gk;
    }
    plist_free(&L);
}

/* Sec. VI-D: partition sizes and distinct inbound counts after every prefix;
 * returns k* (number of moves to apply) and its cumulative gain. */
static int32_t best_prefix(const hg_t *g, const int32_t *rho, int32_t nparts, const move_t *mv,
                           const int32_t *seq, const int64_t *gseq, int32_t M, int32_t omega,
                           int32_t delta, int64_t *best_gain)
{
    plist_t L;
    plist_alloc(g, &L);
    plist_build(g, rho, &L);
    int64_t *sz = xcalloc((size_t)nparts, sizeof(int64_t));
    int64_t *D = xcalloc((size_t)nparts, sizeof(int64_t));
    uint8_t *bad = xcalloc((size_t)nparts, 1);
    for (int32_t v = 0; v < g->n; v++) sz[rho[v]] += g->size[v];
    for (int32_t e = 0; e < g->e; e++)
        for (int32_t i = 0; i < L.len[e]; i++)
            if (L.cin[2 * g->off[e] + i] > 0) D[L.p[2 * g->off[e] + i]]++;
    int64_t nbad = 0;
    for (int32_t p = 0; p < nparts; p++) {
        bad[p] = sz[p] > omega || D[p] > delta;
        nbad += bad[p];
    }
    int64_t cum = 0, bestc = 0;
    int32_t bestk = 0;
    for (int32_t k = 0; k < M; k++) {
        const move_t *x = &mv[seq[k]];
        int32_t v = x->node;
        sz[x->src] -= g->size[v];
        sz[x->dst] += g->size[v];
        for (int64_t t = g->ioff[v]; t < g->ioff[v] + g->nin[v]; t++) {
            int32_t e = g->inc[t];
            int64_t ks = plist_find(g, &L, e, x->src);
            int64_t kd = plist_find_or_add(g, &L, e, x->dst);
            if (--L.cin[ks] == 0) D[x->src]--;
            if (++L.cin[kd] == 1) D[x->dst]++;
        }
        int32_t ps[2] = {x->src, x->dst};
        for (int i = 0; i < 2; i++) {
            int32_t p = ps[i];
            uint8_t b = sz[p] > omega || D[p] > delta;
            nbad += (int64_t)b - bad[p];
            bad[p] = b;
        }
        cum += gseq[k];
        if (nbad == 0 && cum >= bestc) { bestc = cum; bestk = k + 1; }
    }
    plist_free(&L);
    free(sz); free(D); free(bad);
    *best_gain = bestc;
    return bestc > 0 ? bestk : 0;
}

typedef struct {
    int32_t pi, theta, window, rounds, permille, kind, maxlev;
    int32_t lk;   /* 0: C(n) by (eta, id); else K of the learned priority */
    int32_t ll;   /* levels the learned priority ranks (0: all); deeper levels use (eta, id) */
} opts_t;

/* one refinement repetition (Sec. VI); returns the number of moves applied */
static int32_t refine_rep(const hg_t *g, int32_t *rho, int32_t nparts, int second_half, int32_t omega,
                          int32_t delta, const opts_t *o)
{
    plist_t L;
    plist_alloc(g, &L);
    plist_build(g, rho, &L);
    int64_t *psize = xcalloc((size_t)nparts, sizeof(int64_t));
    for (int32_t v = 0; v < g->n; v++) psize[rho[v]] += g->size[v];
    move_t *mv = xcalloc((size_t)g->n + 1, sizeof(move_t));
    int32_t M = propose_moves(g, rho, nparts, &L, psize, omega, second_half, mv);
    plist_free(&L);
    free(psize);
    qsort(mv, (size_t)M, sizeof(move_t), cmp_move);
    int32_t *seq = xcalloc((size_t)M + 1, sizeof(int32_t));
    int64_t *gseq = xcalloc((size_t)M + 1, sizeof(int64_t));
    sequence_moves(g, nparts, mv, M, o->window, o->rounds, seq);
    inseq_gains(g, rho, mv, seq, M, gseq);
    int64_t bg = 0;
    int32_t k = best_prefix(g, rho, nparts, mv, seq, gseq, M, omega, delta, &bg);
    for (int32_t i = 0; i < k; i++) rho[mv[seq[i]].node] = mv[seq[i]].dst;
    free(mv); free(seq); free(gseq);
    return k;
}

/* ------------------------------------------------------------------------ */
/* input checks                                                              */
/* ------------------------------------------------------------------------ */
static void default_opts(opts_t *o)
{
    o->pi = 4; o->theta = 16; o->window = 256; o->rounds = 16; o->permille = 100; o->kind = 0;
    o->maxlev = 256;
    o->lk = 0;
    o->ll = 0;
}

static int read_opts(const int32_t *opt, opts_t *o)
{
    default_opts(o);
    if (opt) {
        o->pi = opt[OPT_PI]; o->theta = opt[OPT_THETA]; o->window = opt[OPT_WINDOW];
        o->rounds = opt[OPT_ROUNDS]; o->permille = opt[OPT_PERMILLE]; o->kind = opt[OPT_KIND];
        o->maxlev = opt[OPT_MAXLEV];
        o->lk = opt[OPT_LK];
        o->ll = opt[OPT_LL];
    }
    if (o->pi < 1 || o->pi > 16 || o->theta < 0 || o->theta > 1024 || o->window < 1 ||
        o->rounds < 0 || o->rounds > 1024 || o->permille < 0 || o->permille > 1000 ||
        (o->kind != 0 && o->kind != 1) || o->maxlev < 0 || o->maxlev > 4096 ||
        (o->lk != 0 && (o->lk < o->pi || o->lk > 16)) || o->ll < 0)
        return OR_ERR_INVALID_ARG;
    return OR_OK;
}

/* Builds the level-0 hypergraph after checking the input. */
static int make_level0(int32_t n, int32_t e, const int32_t *off, const int32_t *pins, const int32_t *nsrc,
                       const int32_t *w, int32_t delta, int32_t kind, hg_t *g)
{
    memset(g, 0, sizeof *g);
    if (off[0] != 0) return OR_ERR_BAD_CSR;
    for (int32_t i = 0; i < e; i++)
        if (off[i + 1] <= off[i]) return OR_ERR_BAD_CSR;
    int64_t np = off[e];
    for (int64_t j = 0; j < np; j++)
        if (pins[j] < 0 || pins[j] >= n) return OR_ERR_BAD_CSR;
    if (nsrc)
        for (int32_t i = 0; i < e; i++)
            if (nsrc[i] < 0 || nsrc[i] > off[i + 1] - off[i]) return OR_ERR_BAD_CSR;
    int32_t *mark = xcalloc((size_t)n + 1, sizeof(int32_t));
    for (int32_t i = 0; i < e; i++)
        for (int64_t j = off[i]; j < off[i + 1]; j++) {
            if (mark[pins[j]] == i + 1) { free(mark); return OR_ERR_BAD_CSR; }
            mark[pins[j]] = i + 1;
        }
    free(mark);
    if (w) {
        int64_t sw = 0;
        for (int32_t i = 0; i < e; i++) {
            if (w[i] < 1 || w[i] > 65536) return OR_ERR_INVALID_ARG;
            sw += w[i];
        }
        if (sw > ((int64_t)1 << 37)) return OR_ERR_INVALID_ARG;
    }
    g->n = n; g->e = e; g->np = np;
    g->off = xcalloc((size_t)e + 1, sizeof(int64_t));
    for (int32_t i = 0; i <= e; i++) g->off[i] = off[i];
    g->pin = xcalloc((size_t)np, sizeof(int32_t));
    memcpy(g->pin, pins, sizeof(int32_t) * (size_t)np);
    g->nsrc = xcalloc((size_t)e, sizeof(int32_t));
    g->w = xcalloc((size_t)e, sizeof(int32_t));
    for (int32_t i = 0; i < e; i++) {
        g->nsrc[i] = kind == 1 ? 0 : (nsrc ? nsrc[i] : 1);
        g->w[i] = w ? w[i] : 1;
    }
    g->size = xcalloc((size_t)n, sizeof(int32_t));
    for (int32_t v = 0; v < n; v++) g->size[v] = 1;
    hg_incidence(g);
    for (int32_t v = 0; v < n; v++)
        if (g->nin[v] > delta) { hg_free(g); return OR_ERR_INFEASIBLE; }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Sec. III: the multilevel driver                                           */
/* ------------------------------------------------------------------------ */
/* model: NULL, or the MD_N-vector of the learned priority (needed when the
 * option learned_k is set) */
int or_partition_ml(int32_t n, int32_t e, const int32_t *off, const int32_t *pins, const int32_t *nsrc,
                    const int32_t *w, int32_t omega, int32_t delta, uint64_t seed, const int32_t *opt,
                    const int32_t *model, int32_t *part_out, int64_t *stats, int64_t *trace)
{
    opts_t o;
    if (n < 0 || e < 0 || omega < 1 || delta < 0 || (n > 0 && !part_out) || (e > 0 && (!off || !pins)))
        return OR_ERR_INVALID_ARG;
    if (read_opts(opt, &o) != OR_OK) return OR_ERR_INVALID_ARG;
    if (o.lk > 0 && (!model || !model_ok(model))) return OR_ERR_INVALID_ARG;
    int32_t zero = 0;
    if (!off) off = &zero;
    hg_t *lv = xcalloc((size_t)o.maxlev + 1, sizeof(hg_t));
    int32_t **gam = xcalloc((size_t)o.maxlev + 1, sizeof(int32_t *));
    int st = make_level0(n, e, off, pins, nsrc, w, delta, o.kind, &lv[0]);
    if (st != OR_OK) { free(lv); free(gam); return st; }
    if (stats) memset(stats, 0, sizeof(int64_t) * ST_N);
    if (trace) memset(trace, 0, sizeof(int64_t) * TR_W * ((size_t)o.maxlev + 1));

    int64_t target_n = ((int64_t)n + omega - 1) / omega;
    int32_t L = 0;
    for (;;) {
        hg_t *g = &lv[L];
        if (trace) { trace[L * TR_W + TR_N] = g->n; trace[L * TR_W + TR_PINS] = g->np; }
        if ((int64_t)g->n <= target_n || L == o.maxlev) break;
        /* the learned priority ranks the top-K lists (K >= Pi); the
         * best-effort pairing takes the nodes with no valid neighbour either way */
        const int learned = o.lk > 0 && (o.ll == 0 || L < o.ll);
        int32_t K = learned ? o.lk : o.pi;
        int32_t *cand = xcalloc((size_t)g->n * K, sizeof(int32_t));
        uint64_t *cs = xcalloc((size_t)g->n * K, sizeof(uint64_t));
        int32_t *mate = xcalloc((size_t)g->n, sizeof(int32_t));
        for (int32_t v = 0; v < g->n; v++) mate[v] = -1;
        propose_pairs(g, L, seed, omega, delta, K, o.permille, cand, cs);
        int64_t nlist = 0;
        for (int32_t v = 0; v < g->n; v++) nlist += cand[(int64_t)v * K] < 0;
        int64_t iso = pair_isolated(g, K, cand, omega, delta, mate);
        if (learned) {
            int32_t *c2 = xcalloc((size_t)g->n * o.pi, sizeof(int32_t));
            uint64_t *s2 = xcalloc((size_t)g->n * o.pi, sizeof(uint64_t));
            learned_candidates(g, L, K, cand, cs, o.pi, model, omega, delta, c2, s2);
            free(cand); free(cs);
            cand = c2;
            cs = s2;
        }
        int64_t r1[3] = {0, 0, 0};
        int64_t pairs = iso + match_all(g->n, o.pi, cand, cs, mate, r1);
        free(cand); free(cs);
        if (trace) {
            int64_t *t = trace + (int64_t)L * TR_W;
            t[TR_PAIRS] = pairs;
            t[TR_ISOPAIRS] = iso;
            t[TR_VALID] = g->n - nlist;
            t[TR_ISOLIST] = nlist;
            t[TR_TGT1] = r1[0];
            t[TR_MAXIN1] = r1[1];
            t[TR_PAIRS1] = r1[2];
        }
        if (pairs == 0) { free(mate); break; }
        gam[L] = xcalloc((size_t)g->n, sizeof(int32_t));
        contract(g, mate, &lv[L + 1], gam[L]);
        free(mate);
        L++;
    }

    /* coarsest clusters are the initial partitions; refine every level */
    int32_t nparts = lv[L].n;
    int32_t *rho = xcalloc((size_t)nparts, sizeof(int32_t));
    for (int32_t v = 0; v < nparts; v++) rho[v] = v;
    int64_t moves_total = 0;
    int32_t half = o.theta / 2;
    for (int32_t l = L; l >= 0; l--) {
        hg_t *g = &lv[l];
        if (l < L) {
            int32_t *r = xcalloc((size_t)g->n, sizeof(int32_t));
            for (int32_t v = 0; v < g->n; v++) r[v] = rho[gam[l][v]];
            free(rho);
            rho = r;
        }
        int64_t moves_l = 0, reps = 0;
        for (int32_t rep = 0; rep < o.theta; rep++) {
            int32_t k = refine_rep(g, rho, nparts, rep >= half, omega, delta, &o);
            reps++;
            moves_l += k;
            if (k == 0) {
                if (rep < half) rep = half - 1;
                else break;
            }
        }
        moves_total += moves_l;
        if (trace) {
            int64_t c, cn;
            objective(g, rho, nparts, &c, &cn);
            trace[l * TR_W + TR_CONN] = c;
            trace[l * TR_W + TR_MOVES] = moves_l;
            trace[l * TR_W + TR_REPS] = reps;
        }
    }

    /* compact partition ids in ascending order of the internal id */
    hg_t *g0 = &lv[0];
    int32_t *newid = xcalloc((size_t)nparts, sizeof(int32_t));
    for (int32_t p = 0; p < nparts; p++) newid[p] = -1;
    for (int32_t v = 0; v < n; v++) newid[rho[v]] = 0;
    int32_t k = 0;
    for (int32_t p = 0; p < nparts; p++)
        if (newid[p] == 0) newid[p] = k++;
    for (int32_t v = 0; v < n; v++) part_out[v] = newid[rho[v]];
    if (stats) {
        int64_t c = 0, cn = 0;
        objective(g0, part_out, k > 0 ? k : 1, &c, &cn);
        int64_t *sz = xcalloc((size_t)k + 1, sizeof(int64_t));
        int64_t *D = xcalloc((size_t)k + 1, sizeof(int64_t));
        int32_t *mark = xcalloc((size_t)k + 1, sizeof(int32_t));
        for (int32_t v = 0; v < n; v++) sz[part_out[v]]++;
        for (int32_t i = 0; i < g0->e; i++)
            for (int64_t j = g0->off[i]; j < g0->off[i + 1]; j++) {
                if (!is_dst_pos(g0, i, j)) continue;
                int32_t p = part_out[g0->pin[j]];
                if (mark[p] != i + 1) { mark[p] = i + 1; D[p]++; }
            }
        int64_t msz = 0, mdist = 0, viol = 0;
        for (int32_t p = 0; p < k; p++) {
            if (sz[p] > msz) msz = sz[p];
            if (D[p] > mdist) mdist = D[p];
            if (sz[p] > omega || D[p] > delta) viol++;
        }
        stats[ST_CONN] = c; stats[ST_CUTNET] = cn; stats[ST_PARTS] = k; stats[ST_MAXSIZE] = msz;
        stats[ST_MAXDIST] = mdist; stats[ST_VIOL] = viol; stats[ST_LEVELS] = L + 1;
        stats[ST_MOVES] = moves_total;
        free(sz); free(D); free(mark);
    }
    if (trace)
        for (int32_t l = 0; l <= L; l++) trace[l * TR_W + TR_PARTS] = k;
    free(newid); free(rho);
    for (int32_t l = 0; l <= L; l++) { hg_free(&lv[l]); free(gam[l]); }
    free(lv); free(gam);
    return OR_OK;
}

int or_partition(int32_t n, int32_t e, const int32_t *off, const int32_t *pins, const int32_t *nsrc,
                 const int32_t *w, int32_t omega, int32_t delta, uint64_t seed, const int32_t *opt,
                 int32_t *part_out, int64_t *stats, int64_t *trace)
{
    return or_partition_ml(n, e, off, pins, nsrc, w, omega, delta, seed, opt, NULL, part_out, stats, trace);
}

/* ------------------------------------------------------------------------ */
/* step-level entry points for the pin tests (one level graph at a time)     */
/* ------------------------------------------------------------------------ */
static void make_level(int32_t n, int32_t e, const int32_t *off, const int32_t *pins, const int32_t *nsrc,
                       const int32_t *w, const int32_t *size, hg_t *g)
{
    memset(g, 0, sizeof *g);
    g->n = n; g->e = e; g->np = e ? off[e] : 0;
    g->off = xcalloc((size_t)e + 1, sizeof(int64_t));
    for (int32_t i = 0; i <= e; i++) g->off[i] = e ? off[i] : 0;
    g->pin = xcalloc((size_t)g->np, sizeof(int32_t));
    if (g->np) memcpy(g->pin, pins, sizeof(int32_t) * (size_t)g->np);
    g->nsrc = xcalloc((size_t)e, sizeof(int32_t));
    g->w = xcalloc((size_t)e, sizeof(int32_t));
    g->size = xcalloc((size_t)n, sizeof(int32_t));
    for (int32_t i = 0; i < e; i++) { g->nsrc[i] = nsrc ? nsrc[i] : 1; g->w[i] = w ? w[i] : 1; }
    for (int32_t v = 0; v < n; v++) g->size[v] = size ? size[v] : 1;
    hg_incidence(g);
}

/* eta(v, .) without noise and inter(v, .) for one node; returns |N(v)|;
 * also returns the noise cap of the level. */
int32_t or_node_histogram(int32_t n, int32_t e, const int32_t *off, const int32_t *pins, const int32_t *nsrc,
                          const int32_t *w, int32_t v, int32_t permille, uint64_t *eta0, int32_t *inter,
                          uint64_t *cap_out)
{
    hg_t g;
    make_level(n, e, off, pins, nsrc, w, NULL, &g);
    uint64_t *q = xcalloc((size_t)e, sizeof(uint64_t));
    uint64_t cap = level_weights(&g, q, permille);
    uint8_t *seen = xcalloc((size_t)n, 1);
    int32_t *nb = xcalloc((size_t)n, sizeof(int32_t));
    memset(eta0, 0, sizeof(uint64_t) * (size_t)n);
    memset(inter, 0, sizeof(int32_t) * (size_t)n);
    int32_t k = node_histogram(&g, q, v, eta0, inter, seen, nb);
    if (cap_out) *cap_out = cap;
    free(q); free(seen); free(nb);
    hg_free(&g);
    return k;
}

uint64_t or_pair_noise(uint64_t seed, int32_t level, int32_t a, int32_t b, uint64_t cap)
{
    return pair_noise(seed, level, a, b, cap);
}

void or_propose(int32_t n, int32_t e, const int32_t *off, const int32_t *pins, const int32_t *nsrc,
                const int32_t *w, const int32_t *size, int32_t omega, int32_t delta, uint64_t seed,
                int32_t level, int32_t pi, int32_t permille, int32_t *cand, uint64_t *cscore)
{
    hg_t g;
    make_level(n, e, off, pins, nsrc, w, size, &g);
    propose_pairs(&g, level, seed, omega, delta, pi, permille, cand, cscore);
    hg_free(&g);
}

int64_t or_pair_isolated(int32_t n, int32_t e, const int32_t *off, const int32_t *pins, const int32_t *nsrc,
                         const int32_t *size, int32_t omega, int32_t delta, int32_t pi, const int32_t *cand,
                         int32_t *mate)
{
    hg_t g;
    make_level(n, e, off, pins, nsrc, NULL, size, &g);
    int64_t r = pair_isolated(&g, pi, cand, omega, delta, mate);
    hg_free(&g);
    return r;
}

int64_t or_match_round(int32_t n, const int32_t *target, const uint64_t *score, int32_t *mate)
{
    return match_round(n, target, score, mate);
}

int64_t or_match_all(int32_t n, int32_t pi, const int32_t *cand, const uint64_t *cscore, int32_t *mate)
{
    return match_all(n, pi, cand, cscore, mate, NULL);
}

/* coarse graph into caller arrays sized n (size_out), e+1 (off_out), e
 * (nsrc_out) and np (pins_out); returns the coarse node count. */
int32_t or_contract(int32_t n, int32_t e, const int32_t *off, const int32_t *pins, const int32_t *nsrc,
                    const int32_t *size, const int32_t *mate, int32_t *gamma, int32_t *size_out,
                    int32_t *off_out, int32_t *pins_out, int32_t *nsrc_out)
{
    hg_t g, c;
    make_level(n, e, off, pins, nsrc, NULL, size, &g);
    contract(&g, mate, &c, gamma);
    memcpy(size_out, c.size, sizeof(int32_t) * (size_t)c.n);
    for (int32_t i = 0; i <= e; i++) off_out[i] = (int32_t)c.off[i];
    if (c.np) memcpy(pins_out, c.pin, sizeof(int32_t) * (size_t)c.np);
    if (e) memcpy(nsrc_out, c.nsrc, sizeof(int32_t) * (size_t)e);
    int32_t nc = c.n;
    hg_free(&g);
    hg_free(&c);
    return nc;
}

void or_objective(int32_t n, int32_t e, const int32_t *off, const int32_t *pins, const int32_t *w,
                  const int32_t *rho, int32_t nparts, int64_t *conn, int64_t *cutnet)
{
    hg_t g;
    make_level(n, e, off, pins, NULL, w, NULL, &g);
    objective(&g, rho, nparts, conn, cutnet);
    hg_free(&g);
}

/* moves in isolation, sorted (p_s asc, gain desc, node asc); returns M */
int32_t or_propose_moves(int32_t n, int32_t e, const int32_t *off, const int32_t *pins, const int32_t *nsrc,
                         const int32_t *w, const int32_t *size, const int32_t *rho, int32_t nparts,
                         int32_t omega, int32_t second_half, int32_t *node, int32_t *src, int32_t *dst,
                         int64_t *gain)
{
    hg_t g;
    make_level(n, e, off, pins, nsrc, w, size, &g);
    plist_t L;
    plist_alloc(&g, &L);
    plist_build(&g, rho, &L);
    int64_t *psize = xcalloc((size_t)nparts, sizeof(int64_t));
    for (int32_t v = 0; v < n; v++) psize[rho[v]] += g.size[v];
    move_t *mv = xcalloc((size_t)n + 1, sizeof(move_t));
    int32_t M = propose_moves(&g, rho, nparts, &L, psize, omega, second_half, mv);
    qsort(mv, (size_t)M, sizeof(move_t), cmp_move);
    for (int32_t i = 0; i < M; i++) { node[i] = mv[i].node; src[i] = mv[i].src; dst[i] = mv[i].dst; gain[i] = mv[i].gain; }
    plist_free(&L);
    free(psize); free(mv);
    hg_free(&g);
    return M;
}

/* moves given sorted; seq_out[k] = index of the k-th move in the sequence */
void or_sequence(int32_t n, int32_t e, const int32_t *off, const int32_t *pins, const int32_t *nsrc,
                 const int32_t *size, int32_t nparts, int32_t M, const int32_t *node, const int32_t *src,
                 const int32_t *dst, const int64_t *gain, int32_t window, int32_t rounds, int32_t *seq_out)
{
    hg_t g;
    make_level(n, e, off, pins, nsrc, NULL, size, &g);
    move_t *mv = xcalloc((size_t)M + 1, sizeof(move_t));
    for (int32_t i = 0; i < M; i++) { mv[i].node = node[i]; mv[i].src = src[i]; mv[i].dst = dst[i]; mv[i].gain = gain[i]; }
    sequence_moves(&g, nparts, mv, M, window, rounds, seq_out);
    free(mv);
    hg_free(&g);
}

/* moves listed in sequence order; gseq_out[k]; returns k* and its gain */
int32_t or_inseq_and_prefix(int32_t n, int32_t e, const int32_t *off, const int32_t *pins, const int32_t *nsrc,
                            const int32_t *w, const int32_t *size, const int32_t *rho, int32_t nparts, int32_t M,
                            const int32_t *node, const int32_t *dst, int32_t omega, int32_t delta,
                            int64_t *gseq_out, int64_t *best_gain)
{
    hg_t g;
    make_level(n, e, off, pins, nsrc, w, size, &g);
    move_t *mv = xcalloc((size_t)M + 1, sizeof(move_t));
    int32_t *seq = xcalloc((size_t)M + 1, sizeof(int32_t));
    for (int32_t i = 0; i < M; i++) {
        mv[i].node = node[i]; mv[i].src = rho[node[i]]; mv[i].dst = dst[i]; mv[i].gain = 0;
        seq[i] = i;
    }
    inseq_gains(&g, rho, mv, seq, M, gseq_out);
    int32_t k = best_prefix(&g, rho, nparts, mv, seq, gseq_out, M, omega, delta, best_gain);
    free(mv); free(seq);
    hg_free(&g);
    return k;
}

/* one refinement repetition on a level graph; rho updated in place */
int32_t or_refine_rep(int32_t n, int32_t e, const int32_t *off, const int32_t *pins, const int32_t *nsrc,
                      const int32_t *w, const int32_t *size, int32_t *rho, int32_t nparts, int32_t second_half,
                      int32_t omega, int32_t delta, int32_t window, int32_t rounds)
{
    hg_t g;
    make_level(n, e, off, pins, nsrc, w, size, &g);
    opts_t o;
    default_opts(&o);
    o.window = window;
    o.rounds = rounds;
    int32_t k = refine_rep(&g, rho, nparts, second_half, omega, delta, &o);
    hg_free(&g);
    return k;
}

/* learned priority: the MLP on count feature rows (16 bytes each) */
int or_mlp_scores(const uint8_t *feat, int64_t count, const int32_t *model, int64_t *out)
{
    if (!model_ok(model)) return OR_ERR_INVALID_ARG;
    for (int64_t i = 0; i < count; i++) out[i] = mlp_score(model, feat + i * ML_IN);
    return OR_OK;
}

/* learned priority on one level: top-K lists in, features of every listed
 * pair (zero rows and rank -1 where the pair is not mutual) and C(n) out */
int or_learned_level(int32_t n, int32_t e, const int32_t *off, const int32_t *pins, const int32_t *nsrc,
                     const int32_t *size, int32_t omega, int32_t delta, int32_t level, int32_t K,
                     const int32_t *candK, const uint64_t *csK, int32_t pi, const int32_t *model, uint8_t *feat,
                     int32_t *rank, int32_t *cand, uint64_t *cscore)
{
    if (!model_ok(model) || K < pi || K > 16) return OR_ERR_INVALID_ARG;
    hg_t g;
    make_level(n, e, off, pins, nsrc, NULL, size, &g);
    uint8_t *emark = xcalloc((size_t)e + 1, 1);
    for (int64_t p = 0; p < (int64_t)n * K; p++) {
        int32_t v = (int32_t)(p / K), j = (int32_t)(p % K), m = candK[p];
        memset(feat + p * ML_IN, 0, ML_IN);
        rank[p] = -1;
        if (m < 0) continue;
        for (int32_t i = 0; i < K; i++)
            if (candK[(int64_t)m * K + i] == v) { rank[p] = i; break; }
        if (rank[p] >= 0) pair_features(&g, level, v, m, csK[p], j, rank[p], omega, delta, emark, feat + p * ML_IN);
    }
    learned_candidates(&g, level, K, candK, csK, pi, model, omega, delta, cand, cscore);
    free(emark);
    hg_free(&g);
    return OR_OK;
}

int32_t or_log_code(uint64_t x) { return log_code(x); }

/* the SplitMix64 output function alone (pinned to the published stream) */
uint64_t or_splitmix64_mix(uint64_t z) { return splitmix64_mix(z); }
