/*
 * CPU oracle for the SQA / PT hot path of Albash, Vinci and Lidar,
 * "Simulated Quantum Annealing Comparison between All-to-All Connectivity
 * Schemes" (arXiv:1603.03755).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, deliberately obvious
 * restatement of what the hot path computes.  Only the tests, the smoke check
 * and the CPU-baseline leg of the benchmark may call it.  It shares no code
 * with the GPU library: it has its own Philox, embeddings, tables and sweeps.
 *
 * Conventions shared with the GPU path *by definition* (each side writes them
 * down on its own):
 *   - spin sigma = +1 <-> bit 0, sigma = -1 <-> bit 1;
 *   - a physical problem is a list of terms, each contributing
 *     w * prod(sigma over its 1..4 members) to the energy;
 *   - Philox4x32-10 keys (seed_lo, seed_hi ^ domain) with the domain words
 *     below;
 *   - the per-attempt uniform u is 32 bits: its high 16 bits come from the
 *     SWEEP_HI stream and its low 16 bits from the SWEEP_LO stream, both at
 *     counter (t, site*Z + z, rho/8, instance), half (rho%8)&1 of output word
 *     (rho%8)/2 (half 0 = bits 0..15);
 *   - acceptance: accept iff x <= 0 or u < T(x), with
 *     T(x) = min(floor(2^32 exp(-x)), 2^32 - 2) for x > 0.
 */
#ifndef SQA_ORACLE_H
#define SQA_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_DOM_INIT 0x6A09E667u
#define ORC_DOM_SWEEP_HI 0xBB67AE85u
#define ORC_DOM_SWEEP_LO 0x3C6EF372u
#define ORC_DOM_SWAP 0xA54FF53Au
#define ORC_DOM_TREE 0x510E527Fu
#define ORC_DOM_WSTART 0x9B05688Cu
#define ORC_DOM_WBOND 0x1F83D9ABu
#define ORC_DOM_WACC 0x5BE0CD19u

/* ---- Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC'11) ---- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* ---- physical problem: sum over terms of w * prod sigma ---- */
typedef struct {
    int32_t n;                 /* physical sites, canonical numbering */
    int32_t n_terms;
    const int32_t *term_size;  /* [n_terms], 1..4 */
    const int32_t *term_mem;   /* [n_terms*4], unused slots -1 */
    const int32_t *term_w;     /* [n_terms] */
    const uint8_t *used;       /* [n] 1 when the site belongs to the embedding */
    const int32_t *colour;     /* [n] graph colour, -1 for unused sites */
    int32_t n_colours;
    const int32_t *inc_ptr;    /* [n+1] CSR: terms that contain each site */
    const int32_t *inc_term;   /* [inc_ptr[n]] */
} orc_problem;

/* Minor embedding of K_N on an Lc x Lc Chimera, Lc = ceil(N/4). */
int32_t orc_me_lc(int32_t N);
int32_t orc_me_n_sites(int32_t N);
int32_t orc_me_n_terms(int32_t N);
int32_t orc_me_site(int32_t Lc, int32_t r, int32_t c, int32_t u, int32_t k);
/* Writes terms, used, colour; chain_sites [N*(Lc+1)] (logical i's chain at
 * i*(Lc+1)); hub [N].  Returns the number of terms. */
int32_t orc_me_build(int32_t N, const int32_t *J, int32_t penalty, int32_t *term_size,
                     int32_t *term_mem, int32_t *term_w, uint8_t *used, int32_t *colour,
                     int32_t *chain_sites, int32_t *hub);

/* LHZ embedding of K_N: K = N(N-1)/2 pair spins, (N-1)(N-2)/2 constraints. */
int32_t orc_lhz_index(int32_t N, int32_t i, int32_t j);
int32_t orc_lhz_n_sites(int32_t N);
int32_t orc_lhz_n_terms(int32_t N);
int32_t orc_lhz_build(int32_t N, const int32_t *J, int32_t lambda, int32_t *term_size,
                      int32_t *term_mem, int32_t *term_w, uint8_t *used, int32_t *colour);

/* Fills inc_ptr [n+1] and inc_term [sum of term sizes]. */
void orc_incidence(int32_t n, int32_t n_terms, const int32_t *term_size,
                   const int32_t *term_mem, int32_t *inc_ptr, int32_t *inc_term);

/* Energy of replica rho of a state stored [n][R]. */
int64_t orc_energy(const orc_problem *pb, const int8_t *s, int32_t R, int32_t rho);
/* Energy change when sigma_site of replica rho flips. */
int64_t orc_flip_delta(const orc_problem *pb, const int8_t *s, int32_t R, int32_t rho,
                       int32_t site);

/* ---- acceptance tables ---- */
double orc_jperp(double beta, double A, int32_t L);
double orc_sqa_x(double alpha, double jperp, int32_t delta, int32_t m);
uint32_t orc_threshold(double x);
/* T[t - t0][(delta - dmin)/2][(m + 2)/2] for even delta in [dmin, dmax]. */
void orc_sqa_table(const double *A, const double *B, double beta, int32_t L, int32_t t0,
                   int32_t t1, int32_t dmin, int32_t dmax, uint32_t *T);
/* T[p][(delta - dmin)/2] with x = beta_p * delta. */
void orc_pt_table(const double *betas, int32_t P, int32_t dmin, int32_t dmax, uint32_t *T);
uint32_t orc_swap_threshold(double beta_p, double beta_q, int64_t dE);

/* ---- random numbers of the chain ---- */
uint32_t orc_sweep_uniform(uint64_t seed, uint32_t t, uint32_t slot, uint32_t rho, uint32_t inst);
uint32_t orc_swap_uniform(uint64_t seed, uint32_t event, uint32_t pair, uint32_t rho, uint32_t inst);
uint32_t orc_tree_draw(uint64_t seed, int32_t inst, int32_t tree, int32_t pos, int32_t N);
/* Initial spins of a state [Z][n][R]; unused sites are +1. */
/* Time-like cluster move streams (see anneal.c).  Start slice of replica
 * rho's cluster at site (canonical index), sweep t: floor(u L / 2^32) with u
 * word rho%4 of WSTART at counter (t, site, rho/4, inst).  Bond uniform of the
 * bond between slices tau and tau+1 (mod L): a 32-bit number whose bit 31-k
 * is bit rho%32 of bit-plane k, plane k being word k%4 of WBOND at counter
 * (t, site*L + tau, (rho/32)*8 + k/4, inst).  Acceptance uniform: word rho%4
 * of WACC at counter (t, site, rho/4, inst). */
uint32_t orc_wolff_start(uint64_t seed, uint32_t t, uint32_t site, uint32_t rho, uint32_t inst, int32_t L);
uint32_t orc_wolff_bond_uniform(uint64_t seed, uint32_t t, uint32_t site, int32_t L, int32_t tau, uint32_t rho,
                                uint32_t inst);
uint32_t orc_wolff_accept_uniform(uint64_t seed, uint32_t t, uint32_t site, uint32_t rho, uint32_t inst);
void orc_init_spins(const orc_problem *pb, int32_t Z, int32_t R, uint64_t seed, int32_t inst,
                    int8_t *s);

/* ---- SQA: path-integral Metropolis sweeps t0..t1-1 on state [L][n][R] ---- */
typedef struct {
    int32_t L;          /* Trotter slices, even, >= 2 */
    int32_t R;          /* replica stride of the state array */
    int32_t S;          /* schedule length */
    double beta;
    const double *A;    /* [S] transverse-field schedule */
    const double *B;    /* [S] problem schedule */
    uint64_t seed;
} orc_sqa_params;
int32_t orc_sqa_run(const orc_problem *pb, const orc_sqa_params *prm, int8_t *s, int32_t inst,
                    int32_t t0, int32_t t1, int32_t rho0, int32_t rho1);
/* Probability threshold of joining two equal neighbouring slices into one
 * time-like cluster: p = 1 - e^(-2 Jperp) = 1 - tanh(beta A / L);
 * 0xFFFFFFFF (always) when A <= 0, else min(floor(2^32 p), 2^32 - 2). */
uint32_t orc_bond_threshold(double beta, double A, int32_t L);
/* The same anneal with one time-like cluster move per (site, replica) per
 * sweep instead of the single-spin sweep. */
int32_t orc_sqa_wolff_run(const orc_problem *pb, const orc_sqa_params *prm, int8_t *s, int32_t inst,
                          int32_t t0, int32_t t1, int32_t rho0, int32_t rho1);

/* ---- PT: sweeps t0..t1-1 on state [P][n][R]; E [P][R] written at exit ---- */
typedef struct {
    int32_t P;
    int32_t R;
    int32_t swap_every;
    const double *betas;  /* [P], strictly decreasing (coldest first) */
    uint64_t seed;
} orc_pt_params;
int32_t orc_pt_run(const orc_problem *pb, const orc_pt_params *prm, int8_t *s, int64_t *E,
                   int32_t inst, int32_t t0, int32_t t1, int32_t rho0, int32_t rho1);

/* ---- decoding (readout of one replica: phys[n] = sigma) ---- */
void orc_me_decode(int32_t N, const int32_t *chain_sites, const int32_t *hub,
                   const int8_t *phys, int8_t *logical);
void orc_prufer_tree(int32_t N, uint64_t seed, int32_t inst, int32_t tree, int32_t *parent);
void orc_star_tree(int32_t N, int32_t *parent);
void orc_chain_tree(int32_t N, int32_t *parent);
void orc_lhz_tree_decode(int32_t N, const int32_t *parent, const int8_t *phys, int8_t *logical);
/* Minimum-weight decoding of an LHZ readout (Sec. IV A): the logical state
 * whose pair products q_i q_j disagree with the fewest pair spins of phys,
 * i.e. the ground state of -sum_{i<j} s_ij q_i q_j.  q_{N-1} = +1; ties go to
 * the first state in binary order (bit i of x set <-> q_i = -1). */
void orc_lhz_mwd_decode(int32_t N, const int8_t *phys, int8_t *logical);
/* Belief-propagation decoding of an LHZ readout (Sec. IV, App. C): pair
 * values p (starting from the readout s) updated `iterations` times, all
 * pairs at once: p_ij <- sign(L0 s_ij + L2 sum_{l != i,j} p_il p_lj), ties
 * keep p_ij, with L0 = ln((1-e)/e) the weight of a reading and
 * L2 = ln(((1-e)^2 + e^2) / (2 e (1-e))) the weight of a two-reading parity
 * check at error rate e; then the spanning tree `parent` reads out the
 * logical state from p (q_0 = +1). */
void orc_lhz_bp_decode(int32_t N, const int8_t *phys, double error_rate, int32_t iterations, const int32_t *parent,
                       int8_t *logical);
void orc_lhz_vote_decode(int32_t N, int32_t n_trees, const int32_t *parents,
                         const int8_t *phys, int8_t *logical);
int64_t orc_logical_energy(int32_t N, const int32_t *J, const int8_t *s);
int64_t orc_ground_energy(int32_t N, const int32_t *J, int8_t *s_best);

#ifdef __cplusplus
}
#endif
#endif
