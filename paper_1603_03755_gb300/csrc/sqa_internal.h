// Internal types of the SQA / PT library: the host-side plan of a problem
// and the plain-old-data records the kernels read.
#pragma once
#include <stdint.h>
#include <vector_types.h>  // uint2

#include <string>
#include <vector>

#include "../../include/sqa.h"

namespace sqa {

constexpr int kMaxTerms = 6;    // terms that contain one site: ME <= 6 couplers,
                                // LHZ one field + <= 4 plaquettes
constexpr int kMaxColours = 4;  // ME 2, LHZ 4
constexpr int kMaxN = 64;       // logical spins
constexpr int kMaxByteWindow = 255;  // per-site threshold window held in one byte

// One term as seen from one of its members: the other members and the
// weight, scaled by the kernel's index stride and carrying its sign.
struct TermRec {
    int16_t p[3];  // other members (compact site index), -1 when absent
    int16_t w;     // K * |weight|, negative when the weight is negative
};

// Everything a sweep needs about one site (60 bytes).
struct SiteRec {
    int16_t nterm;
    int16_t base;     // start of the site's window in a threshold row
    int32_t canon;    // canonical site id: random-number counters, readout
    int32_t lut_off;  // SQA: offset of the site's 2^(nterm+2)-entry table
    TermRec t[kMaxTerms];
};

// A term for energy evaluation: members (compact) and signed weight.
struct ETerm {
    int16_t m[4];   // -1 when absent
    int32_t w;
    int32_t size;
};

// Energy terms of one instance are sorted by weight and size; a class is a
// piece of a run of terms with one weight and one size (runs are cut so that
// the device's counting threads share the work).  Up to kMaxEClasses classes
// per instance.
constexpr int kMaxEClasses = 16;
struct EClass {
    int32_t w;
    int32_t start;
    int32_t count;
    int32_t size;   // spins per term
    int32_t total;  // class 0 only: sum of every term's weight (E of the all-up state)
    int32_t pad_;
};

// Device-side description of one job (one handle) for one launch.
struct JobDev {
    int kind;        // SQA_KIND_SQA or SQA_KIND_PT
    int n;           // used sites (compact numbering, sorted by colour)
    int n_phys;
    int Z;           // L (SQA) or P (PT)
    int W;           // words per (site, z) = ceil(R/32)
    int R;
    int n_inst;
    int ncol;
    int col_ptr[kMaxColours + 1];
    int nrow;        // threshold row length: SQA 3*nd, PT nd
    int n_eterms;
    int swap_every;
    int t0, t1;      // sweeps of this launch
    uint32_t seed_lo;
    uint32_t key_hi;     // seed_hi ^ kDomSweepHi
    uint32_t key_lo;     // seed_hi ^ kDomSweepLo
    uint32_t key_swap;   // seed_hi ^ kDomSwap
    // round keys of the two sweep streams, k + r * Weyl constant for rounds
    // r = 0..9 (first word shared: seed_lo), so the kernels read them from
    // the parameter bank instead of forming them per block
    uint32_t rk0[10], rk_hi[10], rk_lo[10];
    // tie queue of the single-spin sweep in global memory: tieq_stride
    // entries {state word, tie mask} per block (blockIdx.x), at least the
    // items of one colour phase of a block, so the queue cannot fill
    uint2 *tieq;
    int tieq_stride;
    uint32_t *state;     // [I][Z][n][W]
    const SiteRec *sites;    // [I][n]
    const uint32_t *T;       // SQA [S][nrow]; PT [P][nrow]
    const ETerm *eterms;     // [I][n_eterms], sorted by weight and size
    const EClass *ecls;      // [I][kMaxEClasses]; count 0 pads
    const uint32_t *Tsw;     // PT swap thresholds, dE = 1..sw_len[p]
    const int *sw_off;       // [P-1]
    const int *sw_len;       // [P-1]
    int wc;          // words per unit
    int zstride;     // shared-memory words per z row
    int smem_bytes;  // shared memory of one unit
    int lut_entries; // SQA: sum over sites of 2^(nterm+2)
    int use_lut;     // SQA: 1 = per-site code tables, 0 = byte-wise index windows
    int n_ecls;      // weight classes used (max over instances); 0 = too many distinct weights
    int csize;       // blocks per unit (a thread-block cluster when > 1)
    int zr;          // slices (SQA) or slots (PT) per block: Z / csize
    int pairs;       // every term has two spins (minor embedding)
    int task_slices; // single-spin sweep: slices (SQA: slice pairs) or slots per task, 1..4; 0 = the kernel's choice
    // time-like cluster moves (SQA, move == SQA_MOVE_WOLFF)
    int move;
    uint32_t key_wstart, key_wbond, key_wacc;  // seed_hi ^ kDomW*
    const uint32_t *Tb;      // [S] bond thresholds
    const uint32_t *Tacc;    // acceptance thresholds, D/2 = 1..acc_len[t] from acc_off[t]
    const int *acc_off;      // [S]
    const int *acc_len;      // [S]
};

// One unit of work: the words [w0, w0+wc) of one instance of one job.
struct Unit {
    int job;
    int inst;
    int w0;
    int wc;
};

// Host plan of a problem (structure shared by all instances).
struct PlanTerm {
    int size;
    int mem[4];    // canonical members
    int jidx;      // index into J (coupler or LHZ field); -1 for a penalty term
};

struct Plan {
    int emb = 0, N = 0, Lc = 0, n_phys = 0, n = 0, ncol = 0;
    std::vector<int> canon;     // compact -> canonical
    std::vector<int> compact;   // canonical -> compact, -1 unused
    int col_ptr[kMaxColours + 1] = {0, 0, 0, 0, 0};
    std::vector<PlanTerm> terms;
    std::vector<std::vector<int>> site_terms;  // compact site -> term ids
    std::vector<int> chain;     // ME [N][Lc+1] compact, hub first
    std::vector<int> pair;      // LHZ [N][N] compact index of the pair spin
};

// Arguments of the decode kernel.
struct DecodeArgs {
    int method, N, n_trees, Lc;
    const int *chain;         // ME [N][Lc+1] compact, hub first
    const int *pair;          // LHZ [N][N] compact index of the pair spin
    const int *parents;       // [I][n_trees][N]
    const int *orders;        // [I][n_trees][N] breadth-first from vertex 0
    const int32_t *J;         // [I][N(N-1)/2]
    const int64_t *e_ground;  // [I] or null
    int8_t *logical;          // [I][R][N] or null
    int64_t *energy;          // [I][R] or null
    int32_t *success;         // [I] or null (zeroed by the host)
    int bp_iters;             // belief propagation: iterations
    int8_t bp_dec[2][64];     // [reading -1?][S + N - 2]: +1, -1, or 0 (keep)
};

// Builders (host_plan.cpp).
bool build_plan(int emb, int N, Plan &out, std::string &err);
// Per-instance site records and energy terms; S_i written to smax (max over sites).
void build_sites(const Plan &pl, const int32_t *J, int penalty, int K, int smax_all,
                 std::vector<SiteRec> &sites_out);
int site_weight_sum_max(const Plan &pl, const int32_t *J, int penalty);
// Energy terms sorted by weight and size, and their classes; returns the number of
// classes, or 0 when the instance has more than kMaxEClasses distinct weights
// or 4096 or more terms of one weight.
int build_eterms(const Plan &pl, const int32_t *J, int penalty, std::vector<ETerm> &out,
                 std::vector<EClass> &cls);

double jperp(double beta, double A, int L);
double sqa_x(double alpha, double jp, int delta, int m);
uint32_t threshold(double x);
void sqa_tables(const double *A, const double *B, double beta, int L, int S, int dmin, int dmax,
                std::vector<uint32_t> &T);
void pt_tables(const double *betas, int P, int dmin, int dmax, std::vector<uint32_t> &T);
// Time-like cluster move tables: Tb[t] the bond threshold of sweep t
// (floor(2^32 (1 - tanh(beta A_t / L))), 0xFFFFFFFF when A_t = 0), and per
// sweep the acceptance thresholds T(alpha_t D) for D = 2, 4, ... up to
// L * dmax or the first zero (off[t], len[t] into Tacc).
uint32_t bond_threshold(double beta, double A, int L);
void wolff_tables(const double *A, const double *B, double beta, int L, int S, int dmax, std::vector<uint32_t> &Tb,
                  std::vector<uint32_t> &Tacc, std::vector<int> &off, std::vector<int> &len);
void swap_tables(const double *betas, int P, std::vector<uint32_t> &T, std::vector<int> &off,
                 std::vector<int> &len);
// Uniform labelled tree from a Pruefer sequence drawn from the TREE stream:
// parent[v] (parent[0] = -1) and a breadth-first order from vertex 0.
void prufer_tree(int N, uint64_t seed, int inst, int tree, int *parent, int *order);
void star_tree(int N, int *parent, int *order);
void chain_tree(int N, int *parent, int *order);

void set_error(const std::string &msg);

}  // namespace sqa
