/*
 * Embeddings of a fully connected logical Ising problem (Eq. 1 of the paper,
 * H_P = sum_{i<j} J_ij s_i s_j, h = 0) into a physical problem, written as a
 * list of terms w * prod(sigma over members).
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Minor embedding (Sec. II A): K_N on an Lc x Lc Chimera of K_{4,4} cells,
 * Lc = ceil(N/4), each logical spin a chain of Lc+1 physical spins coupled
 * ferromagnetically with -penalty.  The paper shows the layout only as a
 * figure (Fig. 1b); the construction used here is:
 *   site index ((r*Lc + c)*2 + u)*4 + k; u = 0 is the vertical shore
 *   (couples to (r+-1, c), same k), u = 1 the horizontal shore (couples to
 *   (r, c+-1), same k); within a cell every vertical site couples to every
 *   horizontal site.
 *   logical i -> group g = i/4, index m = i%4;
 *   chain(i) = { V(r,g,m) : r <= g }  U  { H(g,c,m) : c >= g };
 *   chain edges V(r,g,m)-V(r+1,g,m) (r<g), H(g,c,m)-H(g,c+1,m) (c>=g),
 *   V(g,g,m)-H(g,g,m), weight -penalty;
 *   logical edge i<j: H(g_i,g_j,m_i)-V(g_i,g_j,m_j) if g_i<g_j,
 *   else V(g,g,m_i)-H(g,g,m_j); weight J_ij.
 *
 * LHZ (Sec. II B, Eq. 2): one physical spin per logical pair (i<j) with local
 * field J_ij, and for every 0 <= i < j <= N-2 a constraint -lambda * prod:
 * the 3-body {(i,i+1),(i,i+2),(i+1,i+2)} when j = i+1, else the 4-body
 * {(i,j),(i,j+1),(i+1,j),(i+1,j+1)}.  There are C(N-1,2) of them.
 *
 * Graph colours (no two members of one term share a colour):
 *   ME:  u xor ((r + c) & 1);  LHZ: 2*(i&1) + (j&1).
 */
#include "oracle.h"

int32_t orc_me_lc(int32_t N) { return (N + 3) / 4; }

int32_t orc_me_n_sites(int32_t N)
{
    int32_t Lc = orc_me_lc(N);
    return 8 * Lc * Lc;
}

int32_t orc_me_n_terms(int32_t N) { return N * (N - 1) / 2 + N * orc_me_lc(N); }

int32_t orc_me_site(int32_t Lc, int32_t r, int32_t c, int32_t u, int32_t k)
{
    return ((r * Lc + c) * 2 + u) * 4 + k;
}

static int32_t pair_index(int32_t N, int32_t i, int32_t j)
{
    /* row-major upper triangle, i < j */
    return i * N - i * (i + 1) / 2 + (j - i - 1);
}

static void put_term(int32_t t, int32_t size, const int32_t *mem, int32_t w, int32_t *term_size,
                     int32_t *term_mem, int32_t *term_w)
{
    term_size[t] = size;
    for (int q = 0; q < 4; q++) term_mem[t * 4 + q] = q < size ? mem[q] : -1;
    term_w[t] = w;
}

int32_t orc_me_build(int32_t N, const int32_t *J, int32_t penalty, int32_t *term_size,
                     int32_t *term_mem, int32_t *term_w, uint8_t *used, int32_t *colour,
                     int32_t *chain_sites, int32_t *hub)
{
    int32_t Lc = orc_me_lc(N);
    int32_t n = orc_me_n_sites(N);
    for (int32_t s = 0; s < n; s++) {
        used[s] = 0;
        colour[s] = -1;
    }
    int32_t t = 0;
    for (int32_t i = 0; i < N; i++) {
        int32_t g = i / 4, m = i % 4, len = 0;
        int32_t *ch = chain_sites + i * (Lc + 1);
        for (int32_t r = 0; r <= g; r++) ch[len++] = orc_me_site(Lc, r, g, 0, m);
        for (int32_t c = g; c < Lc; c++) ch[len++] = orc_me_site(Lc, g, c, 1, m);
        hub[i] = orc_me_site(Lc, g, g, 0, m);
        for (int32_t q = 0; q < len; q++) used[ch[q]] = 1;
        /* chain couplers */
        for (int32_t r = 0; r < g; r++) {
            int32_t mem[2] = {orc_me_site(Lc, r, g, 0, m), orc_me_site(Lc, r + 1, g, 0, m)};
            put_term(t++, 2, mem, -penalty, term_size, term_mem, term_w);
        }
        for (int32_t c = g; c + 1 < Lc; c++) {
            int32_t mem[2] = {orc_me_site(Lc, g, c, 1, m), orc_me_site(Lc, g, c + 1, 1, m)};
            put_term(t++, 2, mem, -penalty, term_size, term_mem, term_w);
        }
        {
            int32_t mem[2] = {orc_me_site(Lc, g, g, 0, m), orc_me_site(Lc, g, g, 1, m)};
            put_term(t++, 2, mem, -penalty, term_size, term_mem, term_w);
        }
    }
    for (int32_t i = 0; i < N; i++)
        for (int32_t j = i + 1; j < N; j++) {
            int32_t gi = i / 4, mi = i % 4, gj = j / 4, mj = j % 4;
            int32_t mem[2];
            if (gi < gj) {
                mem[0] = orc_me_site(Lc, gi, gj, 1, mi);
                mem[1] = orc_me_site(Lc, gi, gj, 0, mj);
            } else {
                mem[0] = orc_me_site(Lc, gi, gi, 0, mi);
                mem[1] = orc_me_site(Lc, gi, gi, 1, mj);
            }
            put_term(t++, 2, mem, J[pair_index(N, i, j)], term_size, term_mem, term_w);
        }
    for (int32_t r = 0; r < Lc; r++)
        for (int32_t c = 0; c < Lc; c++)
            for (int32_t u = 0; u < 2; u++)
                for (int32_t k = 0; k < 4; k++) {
                    int32_t s = orc_me_site(Lc, r, c, u, k);
                    if (used[s]) colour[s] = u ^ ((r + c) & 1);
                }
    return t;
}

int32_t orc_lhz_index(int32_t N, int32_t i, int32_t j) { return pair_index(N, i, j); }

int32_t orc_lhz_n_sites(int32_t N) { return N * (N - 1) / 2; }

int32_t orc_lhz_n_terms(int32_t N) { return N * (N - 1) / 2 + (N - 1) * (N - 2) / 2; }

int32_t orc_lhz_build(int32_t N, const int32_t *J, int32_t lambda, int32_t *term_size,
                      int32_t *term_mem, int32_t *term_w, uint8_t *used, int32_t *colour)
{
    int32_t t = 0;
    for (int32_t i = 0; i < N; i++)
        for (int32_t j = i + 1; j < N; j++) {
            int32_t k = pair_index(N, i, j);
            used[k] = 1;
            colour[k] = 2 * (i & 1) + (j & 1);
            int32_t mem[1] = {k};
            put_term(t++, 1, mem, J[k], term_size, term_mem, term_w);
        }
    for (int32_t i = 0; i + 1 <= N - 2; i++)
        for (int32_t j = i + 1; j <= N - 2; j++) {
            if (j == i + 1) {
                int32_t mem[3] = {pair_index(N, i, i + 1), pair_index(N, i, i + 2),
                                  pair_index(N, i + 1, i + 2)};
                put_term(t++, 3, mem, -lambda, term_size, term_mem, term_w);
            } else {
                int32_t mem[4] = {pair_index(N, i, j), pair_index(N, i, j + 1),
                                  pair_index(N, i + 1, j), pair_index(N, i + 1, j + 1)};
                put_term(t++, 4, mem, -lambda, term_size, term_mem, term_w);
            }
        }
    return t;
}

void orc_incidence(int32_t n, int32_t n_terms, const int32_t *term_size,
                   const int32_t *term_mem, int32_t *inc_ptr, int32_t *inc_term)
{
    for (int32_t s = 0; s <= n; s++) inc_ptr[s] = 0;
    for (int32_t t = 0; t < n_terms; t++)
        for (int32_t q = 0; q < term_size[t]; q++) inc_ptr[term_mem[t * 4 + q] + 1]++;
    for (int32_t s = 0; s < n; s++) inc_ptr[s + 1] += inc_ptr[s];
    /* fill in term order; a cursor per site */
    for (int32_t s = 0; s < n; s++) {
        int32_t pos = inc_ptr[s];
        for (int32_t t = 0; t < n_terms; t++)
            for (int32_t q = 0; q < term_size[t]; q++)
                if (term_mem[t * 4 + q] == s) inc_term[pos++] = t;
    }
}

static int64_t term_value(const orc_problem *pb, int32_t t, const int8_t *s, int32_t R,
                          int32_t rho)
{
    int64_t v = pb->term_w[t];
    for (int32_t q = 0; q < pb->term_size[t]; q++)
        v *= s[(int64_t)pb->term_mem[t * 4 + q] * R + rho];
    return v;
}

int64_t orc_energy(const orc_problem *pb, const int8_t *s, int32_t R, int32_t rho)
{
    int64_t e = 0;
    for (int32_t t = 0; t < pb->n_terms; t++) e += term_value(pb, t, s, R, rho);
    return e;
}

/* Flipping sigma_site negates every term that contains it. */
int64_t orc_flip_delta(const orc_problem *pb, const int8_t *s, int32_t R, int32_t rho,
                       int32_t site)
{
    int64_t before = 0;
    for (int32_t q = pb->inc_ptr[site]; q < pb->inc_ptr[site + 1]; q++)
        before += term_value(pb, pb->inc_term[q], s, R, rho);
    return -2 * before;
}
