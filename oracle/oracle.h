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
 *   - the per-attempt uniform u is 32 bits, u = h * 2^25 + l: h (7 bits) is
 *     the low 7 bits of byte (r/8) of output word (r%4) of the SWEEP_HI
 *     stream at counter (t, site*Z + z, 2*(rho/32) + (r/4)%2, instance),
 *     r = rho%32; l (25 bits) is output word (rho%4) of the SWEEP_LO stream
 *     at counter (t, site*Z + z, rho/4, instance), shifted right by 7;
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

/* Minor embedding of K_N on an Lc x Lc Chimera, Lc = ceil(N/4) (Sec. II A;
 * the layout of Fig. 1b, written out in embed.c): grid size, site count,
 * term count (N(N-1)/2 couplers and N*Lc chain edges) and site index. */
int32_t orc_me_lc(int32_t N);
int32_t orc_me_n_sites(int32_t N);
int32_t orc_me_n_terms(int32_t N);
int32_t orc_me_site(int32_t Lc, int32_t r, int32_t c, int32_t u, int32_t k);
/* The minor-embedded problem (Sec. II A): couplers J_ij between chains and
 * chain edges of weight -penalty.  Writes terms, used, colour; chain_sites
 * [N*(Lc+1)] (logical i's chain at i*(Lc+1)); hub [N].  Returns the number
 * of terms. */
int32_t orc_me_build(int32_t N, const int32_t *J, int32_t penalty, int32_t *term_size,
                     int32_t *term_mem, int32_t *term_w, uint8_t *used, int32_t *colour,
                     int32_t *chain_sites, int32_t *hub);

/* LHZ embedding of K_N (Sec. II B, Eq. 2): K = N(N-1)/2 pair spins with
 * local fields J_ij, (N-1)(N-2)/2 constraints -lambda * prod of 3 or 4 pair
 * spins (Fig. 1c, written out in embed.c): pair index, counts, problem. */
int32_t orc_lhz_index(int32_t N, int32_t i, int32_t j);
int32_t orc_lhz_n_sites(int32_t N);
int32_t orc_lhz_n_terms(int32_t N);
int32_t orc_lhz_build(int32_t N, const int32_t *J, int32_t lambda, int32_t *term_size,
                      int32_t *term_mem, int32_t *term_w, uint8_t *used, int32_t *colour);

/* The terms that contain each site (bookkeeping for the energy change of a
 * flip): fills inc_ptr [n+1] and inc_term [sum of term sizes]. */
void orc_incidence(int32_t n, int32_t n_terms, const int32_t *term_size,
                   const int32_t *term_mem, int32_t *inc_ptr, int32_t *inc_term);

/* Energy of replica rho of a state stored [n][R]: sum over terms of
 * w * prod sigma (Eq. 1 through the embedding, Eq. 2 for LHZ). */
int64_t orc_energy(const orc_problem *pb, const int8_t *s, int32_t R, int32_t rho);
/* Energy change when sigma_site of replica rho flips (the delta of the
 * Metropolis rule, App. B): minus twice the terms that contain the site. */
int64_t orc_flip_delta(const orc_problem *pb, const int8_t *s, int32_t R, int32_t rho,
                       int32_t site);

/* ---- acceptance tables (Eq. 3, App. B; Eq. 9 for the swaps) ---- */
/* Coupling along imaginary time of the Trotter action (the paper defers the
 * action to its references; the standard Suzuki-Trotter form):
 * Jperp = -1/2 ln tanh(beta A / L), infinite when A = 0. */
double orc_jperp(double beta, double A, int32_t L);
/* Exponent of a single-spin flip in that action: x = alpha delta + 2 Jperp m,
 * alpha = beta B / L, m = sigma (sigma_up + sigma_down); Jperp * 0 = 0. */
double orc_sqa_x(double alpha, double jperp, int32_t delta, int32_t m);
/* Metropolis acceptance threshold for exponent x: accept iff x <= 0 or
 * u < T(x) = min(floor(2^32 exp(-x)), 2^32 - 2). */
uint32_t orc_threshold(double x);
/* T[t - t0][(delta - dmin)/2][(m + 2)/2] for even delta in [dmin, dmax]. */
void orc_sqa_table(const double *A, const double *B, double beta, int32_t L, int32_t t0,
                   int32_t t1, int32_t dmin, int32_t dmax, uint32_t *T);
/* PT (App. B): T[p][(delta - dmin)/2] with x = beta_p * delta. */
void orc_pt_table(const double *betas, int32_t P, int32_t dmin, int32_t dmax, uint32_t *T);
/* Replica-exchange threshold (Eq. 9): the exponent (beta_p - beta_q) dE of
 * swapping configurations whose energies differ by dE. */
uint32_t orc_swap_threshold(double beta_p, double beta_q, int64_t dE);

/* ---- random numbers of the chain (Philox streams; the paper only asks for
 * uniform random numbers, so the streams are this implementation's) ---- */
uint32_t orc_sweep_uniform(uint64_t seed, uint32_t t, uint32_t slot, uint32_t rho, uint32_t inst);
uint32_t orc_swap_uniform(uint64_t seed, uint32_t event, uint32_t pair, uint32_t rho, uint32_t inst);
uint32_t orc_tree_draw(uint64_t seed, int32_t inst, int32_t tree, int32_t pos, int32_t N);
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
/* Initial spins of a state [Z][n][R], iid uniform from the INIT stream (the
 * paper does not state the initial state); unused sites are +1. */
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
/* SQA (Eq. 3, App. B, Sec. III): at sweep t, every spin of every slice by
 * colour class with single-spin Metropolis in the Trotter action above. */
int32_t orc_sqa_run(const orc_problem *pb, const orc_sqa_params *prm, int8_t *s, int32_t inst,
                    int32_t t0, int32_t t1, int32_t rho0, int32_t rho1);
/* Probability threshold of joining two equal neighbouring slices into one
 * time-like cluster (Sec. III, Sec. V): p = 1 - e^(-2 Jperp) = 1 - tanh(beta A / L);
 * 0xFFFFFFFF (always) when A <= 0, else min(floor(2^32 p), 2^32 - 2). */
uint32_t orc_bond_threshold(double beta, double A, int32_t L);
/* The same anneal with one time-like (Wolff) cluster move per (site,
 * replica) per sweep instead of the single-spin sweep (Sec. III, Sec. V). */
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
/* Zero-field parallel tempering (App. B, Eq. 9): single-spin Metropolis
 * sweeps at each slot's beta, replica-exchange swaps of neighbouring slots
 * every swap_every sweeps (even and odd pairs in turn). */
int32_t orc_pt_run(const orc_problem *pb, const orc_pt_params *prm, int8_t *s, int64_t *E,
                   int32_t inst, int32_t t0, int32_t t1, int32_t rho0, int32_t rho1);

/* ---- decoding (readout of one replica: phys[n] = sigma) ---- */
/* ME majority vote over each chain (Eq. 4); ties take the chain's hub spin. */
void orc_me_decode(int32_t N, const int32_t *chain_sites, const int32_t *hub,
                   const int8_t *phys, int8_t *logical);
/* Spanning trees of the logical graph for LHZ decoding (App. A): random
 * uniform labelled trees (Pruefer sequences from the TREE stream), the star
 * (Eq. 10) and the chain (Eq. 11). */
void orc_prufer_tree(int32_t N, uint64_t seed, int32_t inst, int32_t tree, int32_t *parent);
void orc_star_tree(int32_t N, int32_t *parent);
void orc_chain_tree(int32_t N, int32_t *parent);
/* LHZ decoding along one tree (App. A): q_0 = +1, a child is its parent times
 * the pair spin between them. */
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
/* Majority vote over n_trees tree decodings (Eq. 5); ties take the first. */
void orc_lhz_vote_decode(int32_t N, int32_t n_trees, const int32_t *parents,
                         const int8_t *phys, int8_t *logical);
/* Logical energy sum_{i<j} J_ij s_i s_j (Eq. 1, h = 0). */
int64_t orc_logical_energy(int32_t N, const int32_t *J, const int8_t *s);
/* Exact logical ground-state energy by enumeration of the 2^(N-1) states
 * with s_{N-1} = +1 (success is reaching it, Sec. III). */
int64_t orc_ground_energy(int32_t N, const int32_t *J, int8_t *s_best);

#ifdef __cplusplus
}
#endif
#endif
