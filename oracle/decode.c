/*
 * Decoding of a physical readout back to a logical state, the logical energy
 * (Eq. 1), and the exact logical ground state by enumeration.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * ME majority vote (Eq. 4): the logical spin is the sign of the sum over its
 * chain.  Chains of even length can tie; a tie takes the value of the chain's
 * hub spin V(g,g,m) (the paper does not say how ties are broken).
 *
 * LHZ spanning-tree decoding (App. A, Eqs. 10-11): fix logical spin 0 to +1
 * and propagate along the tree, the logical value of a child being the parent
 * value times the physical spin of the pair.  The star tree (every spin
 * attached to 0) gives q_i = q_{0,i}; the chain tree gives
 * q_i = prod_{m<i} q_{m,m+1}.  Majority vote over n_T trees (Eq. 5): sign of
 * the sum, ties resolved by the first tree.  Random trees are uniform labelled
 * trees decoded from a Pruefer sequence whose entries are drawn from the TREE
 * stream.
 */
#include <stdlib.h>

#include <math.h>

#include "oracle.h"

void orc_me_decode(int32_t N, const int32_t *chain_sites, const int32_t *hub,
                   const int8_t *phys, int8_t *logical)
{
    int32_t len = orc_me_lc(N) + 1;
    for (int32_t i = 0; i < N; i++) {
        int32_t sum = 0;
        for (int32_t q = 0; q < len; q++) sum += phys[chain_sites[i * len + q]];
        if (sum > 0)
            logical[i] = 1;
        else if (sum < 0)
            logical[i] = -1;
        else
            logical[i] = phys[hub[i]];
    }
}

void orc_star_tree(int32_t N, int32_t *parent)
{
    parent[0] = -1;
    for (int32_t i = 1; i < N; i++) parent[i] = 0;
}

void orc_chain_tree(int32_t N, int32_t *parent)
{
    parent[0] = -1;
    for (int32_t i = 1; i < N; i++) parent[i] = i - 1;
}

/* Root an undirected edge list at vertex 0 (plain breadth-first search). */
static void root_tree(int32_t N, const int32_t *ea, const int32_t *eb, int32_t *parent)
{
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    uint8_t *seen = (uint8_t *)calloc((size_t)N, 1);
    for (int32_t v = 0; v < N; v++) parent[v] = -1;
    int32_t head = 0, tail = 0;
    queue[tail++] = 0;
    seen[0] = 1;
    while (head < tail) {
        int32_t v = queue[head++];
        for (int32_t e = 0; e < N - 1; e++) {
            int32_t w = -1;
            if (ea[e] == v) w = eb[e];
            if (eb[e] == v) w = ea[e];
            if (w >= 0 && !seen[w]) {
                seen[w] = 1;
                parent[w] = v;
                queue[tail++] = w;
            }
        }
    }
    free(queue);
    free(seen);
}

void orc_prufer_tree(int32_t N, uint64_t seed, int32_t inst, int32_t tree, int32_t *parent)
{
    if (N == 1) {
        parent[0] = -1;
        return;
    }
    int32_t *seq = (int32_t *)malloc(sizeof(int32_t) * (size_t)(N > 2 ? N - 2 : 1));
    int32_t *deg = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int32_t *ea = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int32_t *eb = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    for (int32_t q = 0; q < N - 2; q++) seq[q] = (int32_t)orc_tree_draw(seed, inst, tree, q, N);
    for (int32_t v = 0; v < N; v++) deg[v] = 1;
    for (int32_t q = 0; q < N - 2; q++) deg[seq[q]]++;
    int32_t ne = 0;
    for (int32_t q = 0; q < N - 2; q++) {
        int32_t leaf = 0;
        while (deg[leaf] != 1) leaf++; /* smallest current leaf */
        ea[ne] = leaf;
        eb[ne] = seq[q];
        ne++;
        deg[leaf]--;
        deg[seq[q]]--;
    }
    int32_t u = -1, w = -1;
    for (int32_t v = 0; v < N; v++)
        if (deg[v] == 1) {
            if (u < 0)
                u = v;
            else
                w = v;
        }
    ea[ne] = u;
    eb[ne] = w;
    ne++;
    root_tree(N, ea, eb, parent);
    free(seq);
    free(deg);
    free(ea);
    free(eb);
}

void orc_lhz_tree_decode(int32_t N, const int32_t *parent, const int8_t *phys, int8_t *logical)
{
    /* Resolve each vertex by walking to the root: q_v = prod of the pair
     * spins on its path, with q_0 = +1. */
    for (int32_t v = 0; v < N; v++) {
        int32_t val = 1, x = v;
        while (x != 0) {
            int32_t p = parent[x];
            int32_t a = p < x ? p : x, b = p < x ? x : p;
            val *= phys[orc_lhz_index(N, a, b)];
            x = p;
        }
        logical[v] = (int8_t)val;
    }
}

void orc_lhz_mwd_decode(int32_t N, const int8_t *phys, int8_t *logical)
{
    int8_t *q = (int8_t *)malloc((size_t)N);
    int64_t best = 0;
    int have = 0;
    uint64_t count = (uint64_t)1 << (N - 1);
    for (uint64_t x = 0; x < count; x++) {
        for (int32_t i = 0; i < N - 1; i++) q[i] = ((x >> i) & 1) ? -1 : 1;
        q[N - 1] = 1;
        /* agreement of the pair spins with the pair products */
        int64_t score = 0;
        for (int32_t i = 0; i < N; i++)
            for (int32_t j = i + 1; j < N; j++) score += (int64_t)phys[orc_lhz_index(N, i, j)] * q[i] * q[j];
        if (!have || score > best) {
            best = score;
            have = 1;
            for (int32_t i = 0; i < N; i++) logical[i] = q[i];
        }
    }
    free(q);
}

void orc_lhz_bp_decode(int32_t N, const int8_t *phys, double error_rate, int32_t iterations, const int32_t *parent,
                       int8_t *logical)
{
    const double e = error_rate;
    const double L0 = log((1.0 - e) / e);
    const double L2 = log(((1.0 - e) * (1.0 - e) + e * e) / (2.0 * e * (1.0 - e)));
    int8_t *p = (int8_t *)malloc((size_t)N * (size_t)N);
    int8_t *q = (int8_t *)malloc((size_t)N * (size_t)N);
    for (int32_t i = 0; i < N; i++)
        for (int32_t j = 0; j < N; j++)
            p[i * N + j] = i == j ? 1 : phys[orc_lhz_index(N, i < j ? i : j, i < j ? j : i)];
    for (int32_t it = 0; it < iterations; it++) {
        for (int32_t i = 0; i < N; i++)
            for (int32_t j = 0; j < N; j++) {
                if (i == j) {
                    q[i * N + j] = 1;
                    continue;
                }
                int32_t S = 0; /* the N-2 parity checks through a third logical spin */
                for (int32_t l = 0; l < N; l++)
                    if (l != i && l != j) S += p[i * N + l] * p[l * N + j];
                const int32_t s = phys[orc_lhz_index(N, i < j ? i : j, i < j ? j : i)];
                const double d = L0 * (double)s + L2 * (double)S;
                q[i * N + j] = d > 0.0 ? 1 : (d < 0.0 ? -1 : p[i * N + j]);
            }
        int8_t *t = p;
        p = q;
        q = t;
    }
    /* spanning-tree readout of the pair values */
    int8_t *pair = (int8_t *)malloc((size_t)N * (size_t)(N - 1) / 2 + 1);
    for (int32_t i = 0; i < N; i++)
        for (int32_t j = i + 1; j < N; j++) pair[orc_lhz_index(N, i, j)] = p[i * N + j];
    orc_lhz_tree_decode(N, parent, pair, logical);
    free(pair);
    free(p);
    free(q);
}

void orc_lhz_vote_decode(int32_t N, int32_t n_trees, const int32_t *parents,
                         const int8_t *phys, int8_t *logical)
{
    int8_t *tmp = (int8_t *)malloc((size_t)N * (size_t)n_trees);
    for (int32_t t = 0; t < n_trees; t++) orc_lhz_tree_decode(N, parents + t * N, phys, tmp + t * N);
    for (int32_t i = 0; i < N; i++) {
        int32_t sum = 0;
        for (int32_t t = 0; t < n_trees; t++) sum += tmp[t * N + i];
        logical[i] = sum > 0 ? 1 : (sum < 0 ? -1 : tmp[i]);
    }
    free(tmp);
}

int64_t orc_logical_energy(int32_t N, const int32_t *J, const int8_t *s)
{
    int64_t e = 0;
    for (int32_t i = 0; i < N; i++)
        for (int32_t j = i + 1; j < N; j++) e += (int64_t)J[orc_lhz_index(N, i, j)] * s[i] * s[j];
    return e;
}

/* Exact ground state with h = 0: enumerate the 2^(N-1) states with
 * s_{N-1} = +1 (the other half are their global flips), energy from scratch.
 * Returns the minimum; s_best gets the first minimiser in enumeration order. */
int64_t orc_ground_energy(int32_t N, const int32_t *J, int8_t *s_best)
{
    int8_t *s = (int8_t *)malloc((size_t)N);
    int64_t best = 0;
    int have = 0;
    uint64_t count = (uint64_t)1 << (N - 1);
    for (uint64_t x = 0; x < count; x++) {
        for (int32_t i = 0; i < N - 1; i++) s[i] = ((x >> i) & 1) ? -1 : 1;
        s[N - 1] = 1;
        int64_t e = orc_logical_energy(N, J, s);
        if (!have || e < best) {
            best = e;
            have = 1;
            for (int32_t i = 0; i < N; i++) s_best[i] = s[i];
        }
    }
    free(s);
    return best;
}
