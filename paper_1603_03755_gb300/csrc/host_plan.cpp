// Host planning for the SQA / PT library: embeddings (Sec. II A/B of
// arXiv:1603.03755), compact site order by graph colour, per-instance site
// records, acceptance tables and decoding trees.
//
// Compiled with -ffp-contract=off: every double expression below is rounded
// operation by operation, so the thresholds are a fixed function of the
// inputs on any host.
#include <math.h>

#include <algorithm>
#include <numeric>
#include <thread>

#include "philox.cuh"
#include "sqa_internal.h"

namespace sqa {

static int pair_idx(int N, int i, int j) { return i * N - i * (i + 1) / 2 + (j - i - 1); }

// ---------------------------------------------------------------------------
// Minor embedding on Chimera.  K_N on an Lc x Lc grid of K_{4,4} cells,
// Lc = ceil(N/4); each logical spin is a chain of Lc+1 physical spins.  The
// layout (Fig. 1b in the paper) is fixed as follows.  Site id
// ((r*Lc + c)*2 + u)*4 + k.  Logical i -> group g = i/4, slot m = i%4; its
// chain runs down column g on the vertical shore (rows 0..g) and along row g
// on the horizontal shore (columns g..Lc-1), the two halves meeting in cell
// (g, g).  Logical coupler i<j sits in cell (g_i, g_j): horizontal slot m_i
// to vertical slot m_j when g_i < g_j, vertical m_i to horizontal m_j when
// the groups coincide.  Colour: u xor ((r + c) & 1).
// ---------------------------------------------------------------------------
static int chimera(int Lc, int r, int c, int u, int k) { return ((r * Lc + c) * 2 + u) * 4 + k; }

static void plan_me(int N, Plan &pl, std::vector<int> &colour_of)
{
    const int Lc = (N + 3) / 4;
    pl.Lc = Lc;
    pl.n_phys = 8 * Lc * Lc;
    std::vector<char> used(pl.n_phys, 0);
    std::vector<int> chains(N * (Lc + 1));
    for (int i = 0; i < N; i++) {
        const int g = i / 4, m = i % 4;
        int q = 0;
        chains[i * (Lc + 1) + q++] = chimera(Lc, g, g, 0, m);  // hub first
        for (int r = 0; r < g; r++) chains[i * (Lc + 1) + q++] = chimera(Lc, r, g, 0, m);
        for (int c = g; c < Lc; c++) chains[i * (Lc + 1) + q++] = chimera(Lc, g, c, 1, m);
        for (int k = 0; k < Lc + 1; k++) used[chains[i * (Lc + 1) + k]] = 1;
        for (int r = 0; r < g; r++)
            pl.terms.push_back({2, {chimera(Lc, r, g, 0, m), chimera(Lc, r + 1, g, 0, m), -1, -1}, -1});
        for (int c = g; c + 1 < Lc; c++)
            pl.terms.push_back({2, {chimera(Lc, g, c, 1, m), chimera(Lc, g, c + 1, 1, m), -1, -1}, -1});
        pl.terms.push_back({2, {chimera(Lc, g, g, 0, m), chimera(Lc, g, g, 1, m), -1, -1}, -1});
    }
    for (int i = 0; i < N; i++)
        for (int j = i + 1; j < N; j++) {
            const int gi = i / 4, mi = i % 4, gj = j / 4, mj = j % 4;
            PlanTerm t{2, {-1, -1, -1, -1}, pair_idx(N, i, j)};
            if (gi < gj) {
                t.mem[0] = chimera(Lc, gi, gj, 1, mi);
                t.mem[1] = chimera(Lc, gi, gj, 0, mj);
            } else {
                t.mem[0] = chimera(Lc, gi, gi, 0, mi);
                t.mem[1] = chimera(Lc, gi, gi, 1, mj);
            }
            pl.terms.push_back(t);
        }
    colour_of.assign(pl.n_phys, -1);
    for (int s = 0; s < pl.n_phys; s++)
        if (used[s]) {
            const int k = s % 4, u = (s / 4) % 2, cell = s / 8, r = cell / Lc, c = cell % Lc;
            (void)k;
            colour_of[s] = u ^ ((r + c) & 1);
        }
    pl.ncol = 2;
    pl.chain = chains;  // canonical for now; made compact by the caller
}

// ---------------------------------------------------------------------------
// LHZ: one spin per logical pair (field J_ij) and, for 0 <= i < j <= N-2, the
// constraint -lambda * prod over {(i,i+1),(i,i+2),(i+1,i+2)} if j == i+1,
// else over {(i,j),(i,j+1),(i+1,j),(i+1,j+1)}.  Colour 2(i&1) + (j&1).
// ---------------------------------------------------------------------------
static void plan_lhz(int N, Plan &pl, std::vector<int> &colour_of)
{
    pl.n_phys = N * (N - 1) / 2;
    colour_of.assign(pl.n_phys, -1);
    for (int i = 0; i < N; i++)
        for (int j = i + 1; j < N; j++) {
            const int k = pair_idx(N, i, j);
            colour_of[k] = 2 * (i & 1) + (j & 1);
            pl.terms.push_back({1, {k, -1, -1, -1}, k});
        }
    for (int i = 0; i <= N - 3; i++)
        for (int j = i + 1; j <= N - 2; j++) {
            if (j == i + 1)
                pl.terms.push_back({3, {pair_idx(N, i, i + 1), pair_idx(N, i, i + 2),
                                        pair_idx(N, i + 1, i + 2), -1}, -1});
            else
                pl.terms.push_back({4, {pair_idx(N, i, j), pair_idx(N, i, j + 1),
                                        pair_idx(N, i + 1, j), pair_idx(N, i + 1, j + 1)}, -1});
        }
    pl.ncol = 4;
}

bool build_plan(int emb, int N, Plan &pl, std::string &err)
{
    pl = Plan();
    pl.emb = emb;
    pl.N = N;
    std::vector<int> colour_of;
    if (emb == SQA_EMB_ME_CHIMERA)
        plan_me(N, pl, colour_of);
    else if (emb == SQA_EMB_LHZ)
        plan_lhz(N, pl, colour_of);
    else {
        err = "unknown embedding";
        return false;
    }
    // compact numbering: used sites sorted by (colour, canonical id)
    std::vector<int> order;
    for (int s = 0; s < pl.n_phys; s++)
        if (colour_of[s] >= 0) order.push_back(s);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return colour_of[a] < colour_of[b]; });
    pl.n = (int)order.size();
    pl.canon = order;
    pl.compact.assign(pl.n_phys, -1);
    for (int i = 0; i < pl.n; i++) pl.compact[order[i]] = i;
    for (int c = 0; c <= kMaxColours; c++) pl.col_ptr[c] = 0;
    for (int i = 0; i < pl.n; i++) pl.col_ptr[colour_of[order[i]] + 1]++;
    for (int c = 0; c < kMaxColours; c++) pl.col_ptr[c + 1] += pl.col_ptr[c];
    for (int c = pl.ncol + 1; c <= kMaxColours; c++) pl.col_ptr[c] = pl.col_ptr[pl.ncol];
    pl.site_terms.assign(pl.n, {});
    for (int t = 0; t < (int)pl.terms.size(); t++)
        for (int q = 0; q < pl.terms[t].size; q++) pl.site_terms[pl.compact[pl.terms[t].mem[q]]].push_back(t);
    for (int i = 0; i < pl.n; i++)
        if ((int)pl.site_terms[i].size() > kMaxTerms) {
            err = "a site has more terms than supported";
            return false;
        }
    if (emb == SQA_EMB_ME_CHIMERA) {
        for (auto &c : pl.chain) c = pl.compact[c];
    } else {
        pl.pair.assign(N * N, -1);
        for (int i = 0; i < N; i++)
            for (int j = i + 1; j < N; j++) {
                const int c = pl.compact[pair_idx(N, i, j)];
                pl.pair[i * N + j] = c;
                pl.pair[j * N + i] = c;
            }
    }
    return true;
}

static int term_weight(const PlanTerm &t, const int32_t *J, int penalty)
{
    return t.jidx >= 0 ? J[t.jidx] : -penalty;
}

int site_weight_sum_max(const Plan &pl, const int32_t *J, int penalty)
{
    int smax = 0;
    for (int i = 0; i < pl.n; i++) {
        int s = 0;
        for (int t : pl.site_terms[i]) s += std::abs(term_weight(pl.terms[t], J, penalty));
        smax = std::max(smax, s);
    }
    return smax;
}

// Site i's flip changes the energy by delta = -2 S_i + 4 U where S_i is the
// sum of |w| over its terms and U the |w|-weighted count of terms whose value
// is currently negative (they turn positive).  The kernels index a threshold
// row with base + K*U (+ the temporal part for SQA); base aligns the site's
// window so that delta lands on (delta - dmin)/2 with dmin = -2 smax_all.
void build_sites(const Plan &pl, const int32_t *J, int penalty, int K, int smax_all,
                 std::vector<SiteRec> &out)
{
    out.assign(pl.n, SiteRec{});
    int lut = 0;
    for (int i = 0; i < pl.n; i++) {
        SiteRec &r = out[i];
        r.nterm = (int16_t)pl.site_terms[i].size();
        r.canon = pl.canon[i];
        r.lut_off = lut;
        lut += 1 << (r.nterm + 2);
        int S = 0;
        for (int q = 0; q < kMaxTerms; q++) {
            TermRec &tr = r.t[q];
            tr.p[0] = tr.p[1] = tr.p[2] = -1;
            tr.w = 0;
            if (q >= r.nterm) continue;
            const PlanTerm &t = pl.terms[pl.site_terms[i][q]];
            const int w = term_weight(t, J, penalty);
            S += std::abs(w);
            int np = 0;
            for (int k = 0; k < t.size; k++) {
                const int c = pl.compact[t.mem[k]];
                if (c != i) tr.p[np++] = (int16_t)c;
            }
            tr.w = (int16_t)(w < 0 ? -K * std::abs(w) : K * std::abs(w));
        }
        // SQA (K = 6): row index 3*((delta - dmin)/2) + (m+2)/2
        //             = 3*(smax - S_i) + 6U + 2 - tc;  PT (K = 2): (smax - S_i) + 2U.
        r.base = (int16_t)(K == 6 ? 3 * (smax_all - S) : (smax_all - S));
    }
}

int build_eterms(const Plan &pl, const int32_t *J, int penalty, std::vector<ETerm> &out,
                 std::vector<EClass> &cls)
{
    out.clear();
    for (const PlanTerm &t : pl.terms) {
        ETerm e;
        for (int k = 0; k < 4; k++) e.m[k] = (int16_t)(k < t.size ? pl.compact[t.mem[k]] : -1);
        e.w = term_weight(t, J, penalty);
        e.size = t.size;
        out.push_back(e);
    }
    std::stable_sort(out.begin(), out.end(),
                     [](const ETerm &a, const ETerm &b) { return a.w != b.w ? a.w < b.w : a.size < b.size; });
    // runs of equal weight and size
    std::vector<EClass> runs;
    int total = 0;
    for (size_t q = 0; q < out.size(); q++) {
        total += out[q].w;
        if (q == 0 || out[q].w != out[q - 1].w || out[q].size != out[q - 1].size)
            runs.push_back(EClass{out[q].w, (int32_t)q, 0, out[q].size, 0, 0});
        runs.back().count++;
    }
    cls.assign(kMaxEClasses, EClass{0, 0, 0, 0, 0, 0});
    cls[0].total = total;
    const int nw = (int)runs.size();
    bool fits = nw <= kMaxEClasses;
    for (const EClass &r : runs) fits = fits && r.count < 4096;  // 12-plane counters on the device
    if (!fits) return 0;
    if (nw == 0) return 0;
    // cut the runs into pieces of at most `chunk` terms, as many pieces as
    // the table holds, so that the device's counting threads share the work:
    // sum ceil(c / chunk) <= n_terms / chunk + nw <= kMaxEClasses
    const int nt = (int)out.size();
    const int room = kMaxEClasses - nw;
    const int chunk = room > 0 ? std::max(16, (nt + room - 1) / room) : nt;
    int nc = 0;
    for (const EClass &r : runs)
        for (int q = 0; q < r.count; q += chunk) cls[nc++] = EClass{r.w, r.start + q, std::min(chunk, r.count - q), r.size, 0, 0};
    cls[0].total = total;
    return nc;
}

// ---------------------------------------------------------------------------
// Acceptance thresholds.  SQA (discrete-time path integral of Eq. 3 with L
// Trotter slices): flipping sigma_i^tau changes the action by
// x = alpha*delta + 2*Jperp*m with alpha = beta*B/L,
// Jperp = -1/2 ln tanh(beta*A/L), m = sigma_i^tau (sigma_i^{tau-1} +
// sigma_i^{tau+1}).  Accept iff x <= 0 or u < T(x),
// T(x) = min(floor(2^32 e^-x), 2^32 - 2); x <= 0 is stored as 2^32 - 1 so
// that min(u, 2^32 - 2) < T is the whole test.
// ---------------------------------------------------------------------------
double jperp(double beta, double A, int L)
{
    const double a = beta * A / (double)L;
    if (a <= 0.0) return INFINITY;
    return -0.5 * log(tanh(a));
}

double sqa_x(double alpha, double jp, int delta, int m)
{
    const double xa = alpha * (double)delta;
    const double xt = (m == 0) ? 0.0 : 2.0 * jp * (double)m;
    return xa + xt;
}

uint32_t threshold(double x)
{
    if (x <= 0.0) return 0xFFFFFFFFu;
    // 2^32 e^-x < 0.44 for x >= 23, so the floor is 0 whatever the last bit
    // of exp: skip the call
    if (x >= 23.0) return 0u;
    const double v = floor(ldexp(exp(-x), 32));
    if (v >= 4294967294.0) return 0xFFFFFFFEu;
    return (uint32_t)v;
}

void sqa_tables(const double *A, const double *B, double beta, int L, int S, int dmin, int dmax,
                std::vector<uint32_t> &T)
{
    const int nd = (dmax - dmin) / 2 + 1;
    T.assign((size_t)S * nd * 3, 0);
    auto rows = [&](int t0, int t1) {
        for (int t = t0; t < t1; t++) {
            const double alpha = beta * B[t] / (double)L;
            const double jp = jperp(beta, A[t], L);
            for (int di = 0; di < nd; di++)
                for (int mi = 0; mi < 3; mi++)
                    T[((size_t)t * nd + di) * 3 + mi] = threshold(sqa_x(alpha, jp, dmin + 2 * di, 2 * mi - 2));
        }
    };
    // rows are independent: large tables are built by several host threads
    const int64_t work = (int64_t)S * nd * 3;
    int nthr = (int)std::min<unsigned>(std::max(1u, std::thread::hardware_concurrency()), 16u);
    if (work < (1 << 20)) nthr = 1;
    if (nthr == 1) {
        rows(0, S);
        return;
    }
    std::vector<std::thread> pool;
    for (int k = 0; k < nthr; k++) {
        const int t0 = (int)((int64_t)S * k / nthr), t1 = (int)((int64_t)S * (k + 1) / nthr);
        pool.emplace_back(rows, t0, t1);
    }
    for (auto &th : pool) th.join();
}

uint32_t bond_threshold(double beta, double A, int L)
{
    const double a = beta * A / (double)L;
    if (a <= 0.0) return 0xFFFFFFFFu;
    const double v = floor(ldexp(1.0 - tanh(a), 32));
    if (v >= 4294967294.0) return 0xFFFFFFFEu;
    return (uint32_t)v;
}

void wolff_tables(const double *A, const double *B, double beta, int L, int S, int dmax, std::vector<uint32_t> &Tb,
                  std::vector<uint32_t> &Tacc, std::vector<int> &off, std::vector<int> &len)
{
    Tb.assign(S, 0);
    off.assign(S, 0);
    len.assign(S, 0);
    const int64_t half_max = (int64_t)L * std::max(dmax, 0) / 2;  // D/2 of the largest cluster change
    // rows are independent: split the sweeps over host threads, then join
    int nthr = (int)std::min<unsigned>(std::max(1u, std::thread::hardware_concurrency()), 16u);
    if ((int64_t)S * std::min<int64_t>(half_max, 64) < (1 << 16)) nthr = 1;
    std::vector<std::vector<uint32_t>> part(nthr);
    auto rows = [&](int k, int t0, int t1) {
        for (int t = t0; t < t1; t++) {
            Tb[t] = bond_threshold(beta, A[t], L);
            const double alpha = beta * B[t] / (double)L;
            int n = 0;
            for (int64_t d = 1; d <= half_max; d++) {
                const uint32_t T = threshold(alpha * (double)(2 * d));
                if (T == 0) break;
                part[k].push_back(T);
                n++;
            }
            len[t] = n;
        }
    };
    std::vector<std::thread> pool;
    std::vector<int> t_lo(nthr + 1);
    for (int k = 0; k <= nthr; k++) t_lo[k] = (int)((int64_t)S * k / nthr);
    if (nthr == 1)
        rows(0, 0, S);
    else {
        for (int k = 0; k < nthr; k++) pool.emplace_back(rows, k, t_lo[k], t_lo[k + 1]);
        for (auto &th : pool) th.join();
    }
    Tacc.clear();
    for (int k = 0; k < nthr; k++) Tacc.insert(Tacc.end(), part[k].begin(), part[k].end());
    int o = 0;
    for (int t = 0; t < S; t++) {
        off[t] = o;
        o += len[t];
    }
    if (Tacc.empty()) Tacc.push_back(0);  // keep one element so the upload is never empty
}

void pt_tables(const double *betas, int P, int dmin, int dmax, std::vector<uint32_t> &T)
{
    const int nd = (dmax - dmin) / 2 + 1;
    T.assign((size_t)P * nd, 0);
    for (int p = 0; p < P; p++)
        for (int di = 0; di < nd; di++) T[(size_t)p * nd + di] = threshold(betas[p] * (double)(dmin + 2 * di));
}

// Swap of slots p, p+1 (Eq. 9): accept iff dE = E_{p+1} - E_p <= 0 or
// u < T((beta_p - beta_{p+1}) dE).  Stored for dE = 1 .. len_p, the last dE
// whose threshold is non-zero (T is non-increasing in dE).
void swap_tables(const double *betas, int P, std::vector<uint32_t> &T, std::vector<int> &off,
                 std::vector<int> &len)
{
    T.clear();
    off.assign(std::max(P - 1, 1), 0);
    len.assign(std::max(P - 1, 1), 0);
    for (int p = 0; p + 1 < P; p++) {
        const double db = betas[p] - betas[p + 1];
        off[p] = (int)T.size();
        int n = 0;
        for (int64_t dE = 1; dE <= (1 << 22); dE++) {
            const uint32_t v = threshold(db * (double)dE);
            if (v == 0) break;
            T.push_back(v);
            n++;
        }
        len[p] = n;
    }
    if (T.empty()) T.push_back(0);
}

// ---------------------------------------------------------------------------
// Decoding trees (App. A).  Random trees: entry q of tree t's Pruefer
// sequence is floor(x * N / 2^32), x = word 0 of the TREE stream at counter
// (t, q, 0, instance).
// ---------------------------------------------------------------------------
static void bfs_order(int N, const std::vector<std::vector<int>> &adj, int *parent, int *order)
{
    std::vector<char> seen(N, 0);
    int head = 0, tail = 0;
    order[tail++] = 0;
    seen[0] = 1;
    parent[0] = -1;
    while (head < tail) {
        const int v = order[head++];
        std::vector<int> nb = adj[v];
        std::sort(nb.begin(), nb.end());
        for (int w : nb)
            if (!seen[w]) {
                seen[w] = 1;
                parent[w] = v;
                order[tail++] = w;
            }
    }
}

void prufer_tree(int N, uint64_t seed, int inst, int tree, int *parent, int *order)
{
    std::vector<std::vector<int>> adj(N);
    if (N >= 2) {
        std::vector<int> seq(std::max(N - 2, 0)), deg(N, 1);
        const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32) ^ kDomTree;
        for (int q = 0; q < N - 2; q++) {
            const U4 v = philox((uint32_t)tree, (uint32_t)q, 0u, (uint32_t)inst, k0, k1);
            seq[q] = (int)(((uint64_t)v.x * (uint64_t)N) >> 32);
            deg[seq[q]]++;
        }
        for (int q = 0; q < N - 2; q++) {
            int leaf = 0;
            while (deg[leaf] != 1) leaf++;
            adj[leaf].push_back(seq[q]);
            adj[seq[q]].push_back(leaf);
            deg[leaf]--;
            deg[seq[q]]--;
        }
        int a = -1, b = -1;
        for (int v = 0; v < N; v++)
            if (deg[v] == 1) (a < 0 ? a : b) = v;
        adj[a].push_back(b);
        adj[b].push_back(a);
    }
    bfs_order(N, adj, parent, order);
}

void star_tree(int N, int *parent, int *order)
{
    parent[0] = -1;
    for (int i = 0; i < N; i++) order[i] = i;
    for (int i = 1; i < N; i++) parent[i] = 0;
}

void chain_tree(int N, int *parent, int *order)
{
    parent[0] = -1;
    for (int i = 0; i < N; i++) order[i] = i;
    for (int i = 1; i < N; i++) parent[i] = i - 1;
}

}  // namespace sqa
