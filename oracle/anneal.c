/*
 * Simulated quantum annealing (discrete-time path-integral Monte Carlo) and
 * parallel tempering, single-spin Metropolis, one replica at a time.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * SQA (Eq. 3, H(t) = A(t) H_X + B(t) H_P with H_X = -sum sigma^x; App. B,
 * fixed Trotter slicing).  The paper defers the Trotter action to its
 * references; the standard Suzuki-Trotter form with periodic imaginary time
 * is used:  weight ~ exp(-alpha sum_tau E_P(sigma^tau)
 *                        + Jperp sum_tau sum_i sigma_i^tau sigma_i^{tau+1}),
 * alpha = beta B / L, Jperp = -1/2 ln tanh(beta A / L).  Flipping sigma_i^tau
 * changes the exponent by -x with x = alpha*delta + 2*Jperp*m, where delta is
 * the change of E_P and m = sigma_i^tau (sigma_i^{tau-1} + sigma_i^{tau+1}).
 *
 * PT (App. B): P replicas of the classical problem at inverse temperatures
 * beta_p; single-spin Metropolis sweeps (x = beta_p * delta); every
 * swap_every sweeps neighbouring slots (p, p+1) exchange configurations with
 * probability min{1, exp[(E_{p+1} - E_p)(beta_{p+1} - beta_p)]} (Eq. 9).
 *
 * Sweep order: colour classes ascending (SQA: class 2*colour + (tau&1)),
 * then site, slice (or slot) and replica ascending.  Sites of one class do not
 * interact, so this order fixes the result.
 */
#include <math.h>

#include "oracle.h"

double orc_jperp(double beta, double A, int32_t L)
{
    double a = beta * A / (double)L;
    if (a <= 0.0) return INFINITY;
    return -0.5 * log(tanh(a));
}

double orc_sqa_x(double alpha, double jperp, int32_t delta, int32_t m)
{
    double xa = alpha * (double)delta;
    double xt;
    if (m == 0)
        xt = 0.0; /* the temporal term vanishes, also when Jperp is infinite */
    else
        xt = 2.0 * jperp * (double)m;
    return xa + xt;
}

uint32_t orc_threshold(double x)
{
    if (x <= 0.0) return 0xFFFFFFFFu;
    double v = floor(ldexp(exp(-x), 32));
    if (v >= 4294967294.0) return 0xFFFFFFFEu;
    return (uint32_t)v;
}

void orc_sqa_table(const double *A, const double *B, double beta, int32_t L, int32_t t0,
                   int32_t t1, int32_t dmin, int32_t dmax, uint32_t *T)
{
    int32_t nd = (dmax - dmin) / 2 + 1;
    for (int32_t t = t0; t < t1; t++) {
        double alpha = beta * B[t] / (double)L;
        double jp = orc_jperp(beta, A[t], L);
        for (int32_t di = 0; di < nd; di++)
            for (int32_t mi = 0; mi < 3; mi++) {
                int32_t delta = dmin + 2 * di, m = 2 * mi - 2;
                T[((int64_t)(t - t0) * nd + di) * 3 + mi] = orc_threshold(orc_sqa_x(alpha, jp, delta, m));
            }
    }
}

void orc_pt_table(const double *betas, int32_t P, int32_t dmin, int32_t dmax, uint32_t *T)
{
    int32_t nd = (dmax - dmin) / 2 + 1;
    for (int32_t p = 0; p < P; p++)
        for (int32_t di = 0; di < nd; di++)
            T[(int64_t)p * nd + di] = orc_threshold(betas[p] * (double)(dmin + 2 * di));
}

uint32_t orc_swap_threshold(double beta_p, double beta_q, int64_t dE)
{
    double dbeta = beta_p - beta_q;
    return orc_threshold(dbeta * (double)dE);
}

static int8_t *at(int8_t *s, int32_t n, int32_t R, int32_t z, int32_t site, int32_t rho)
{
    return s + ((int64_t)z * n + site) * R + rho;
}

int32_t orc_sqa_run(const orc_problem *pb, const orc_sqa_params *prm, int8_t *s, int32_t inst,
                    int32_t t0, int32_t t1, int32_t rho0, int32_t rho1)
{
    int32_t L = prm->L, R = prm->R, n = pb->n;
    if (L < 2 || (L & 1) || t0 < 0 || t1 > prm->S || rho0 < 0 || rho1 > R) return -1;
    for (int32_t t = t0; t < t1; t++) {
        double alpha = prm->beta * prm->B[t] / (double)L;
        double jp = orc_jperp(prm->beta, prm->A[t], L);
        for (int32_t cls = 0; cls < 2 * pb->n_colours; cls++) {
            int32_t chi = cls / 2, parity = cls % 2;
            for (int32_t site = 0; site < n; site++) {
                if (!pb->used[site] || pb->colour[site] != chi) continue;
                for (int32_t tau = parity; tau < L; tau += 2) {
                    int8_t *slice = s + (int64_t)tau * n * R;
                    int32_t up = (tau + L - 1) % L, dn = (tau + 1) % L;
                    for (int32_t rho = rho0; rho < rho1; rho++) {
                        int32_t sig = *at(s, n, R, tau, site, rho);
                        int32_t delta = (int32_t)orc_flip_delta(pb, slice, R, rho, site);
                        int32_t m = sig * (*at(s, n, R, up, site, rho) + *at(s, n, R, dn, site, rho));
                        double x = orc_sqa_x(alpha, jp, delta, m);
                        uint32_t u = orc_sweep_uniform(prm->seed, (uint32_t)t,
                                                       (uint32_t)(site * L + tau), (uint32_t)rho,
                                                       (uint32_t)inst);
                        if (x <= 0.0 || u < orc_threshold(x)) *at(s, n, R, tau, site, rho) = (int8_t)-sig;
                    }
                }
            }
        }
    }
    return 0;
}

uint32_t orc_bond_threshold(double beta, double A, int32_t L)
{
    double a = beta * A / (double)L;
    if (a <= 0.0) return 0xFFFFFFFFu;
    double v = floor(ldexp(1.0 - tanh(a), 32));
    if (v >= 4294967294.0) return 0xFFFFFFFEu;
    return (uint32_t)v;
}

/* Time-like cluster move (Sec. III, App. B: one cluster update along
 * imaginary time per spatial site and sweep).  For replica rho of a site:
 * a start slice tau0 is drawn; the cluster grows forward from tau0 through
 * each bond (tau, tau+1) whose two slices carry equal spins and whose bond
 * uniform is below the bond threshold (probability 1 - e^(-2 Jperp)), and
 * stops at the first bond that does not join; it then grows backward from
 * tau0 the same way, never past the forward end (at most L slices).  The
 * temporal part of the action is accounted for by this construction, so the
 * cluster is flipped with the Metropolis test on the problem part alone:
 * accept iff x <= 0 or u < T(x), x = alpha * D, D the sum of the flip
 * energies of the site over the cluster's slices (all taken before the flip;
 * the site's terms lie within one slice).  Sites of one colour do not share a
 * term, so a colour class moves in any order. */
int32_t orc_sqa_wolff_run(const orc_problem *pb, const orc_sqa_params *prm, int8_t *s, int32_t inst,
                          int32_t t0, int32_t t1, int32_t rho0, int32_t rho1)
{
    int32_t L = prm->L, R = prm->R, n = pb->n;
    if (L < 2 || (L & 1) || t0 < 0 || t1 > prm->S || rho0 < 0 || rho1 > R) return -1;
    for (int32_t t = t0; t < t1; t++) {
        double alpha = prm->beta * prm->B[t] / (double)L;
        uint32_t Tb = orc_bond_threshold(prm->beta, prm->A[t], L);
        for (int32_t chi = 0; chi < pb->n_colours; chi++)
            for (int32_t site = 0; site < n; site++) {
                if (!pb->used[site] || pb->colour[site] != chi) continue;
                for (int32_t rho = rho0; rho < rho1; rho++) {
                    int32_t tau0 = (int32_t)orc_wolff_start(prm->seed, (uint32_t)t, (uint32_t)site, (uint32_t)rho,
                                                            (uint32_t)inst, L);
                    /* bond (tau, tau+1 mod L) joins */
#define ORC_JOINS(tau)                                                                                 \
    (*at(s, n, R, (tau), site, rho) == *at(s, n, R, ((tau) + 1) % L, site, rho) &&                      \
     (Tb == 0xFFFFFFFFu ||                                                                             \
      orc_wolff_bond_uniform(prm->seed, (uint32_t)t, (uint32_t)site, L, (tau), (uint32_t)rho, (uint32_t)inst) < Tb))
                    int32_t fwd = 0;
                    while (fwd < L - 1 && ORC_JOINS((tau0 + fwd) % L)) fwd++;
                    int32_t back = 0;
                    while (back < L - 1 - fwd && ORC_JOINS((tau0 - 1 - back + 2 * L) % L)) back++;
#undef ORC_JOINS
                    int64_t D = 0;
                    for (int32_t q = -back; q <= fwd; q++) {
                        int32_t tau = (tau0 + q + L) % L;
                        D += orc_flip_delta(pb, s + (int64_t)tau * n * R, R, rho, site);
                    }
                    double x = alpha * (double)D;
                    uint32_t u = orc_wolff_accept_uniform(prm->seed, (uint32_t)t, (uint32_t)site, (uint32_t)rho,
                                                          (uint32_t)inst);
                    if (x <= 0.0 || u < orc_threshold(x))
                        for (int32_t q = -back; q <= fwd; q++) {
                            int8_t *v = at(s, n, R, (tau0 + q + L) % L, site, rho);
                            *v = (int8_t)-*v;
                        }
                }
            }
    }
    return 0;
}

static void pt_energies(const orc_problem *pb, const int8_t *s, int32_t P, int32_t R,
                        int32_t rho0, int32_t rho1, int64_t *E)
{
    for (int32_t p = 0; p < P; p++)
        for (int32_t rho = rho0; rho < rho1; rho++)
            E[(int64_t)p * R + rho] = orc_energy(pb, s + (int64_t)p * pb->n * R, R, rho);
}

int32_t orc_pt_run(const orc_problem *pb, const orc_pt_params *prm, int8_t *s, int64_t *E,
                   int32_t inst, int32_t t0, int32_t t1, int32_t rho0, int32_t rho1)
{
    int32_t P = prm->P, R = prm->R, n = pb->n;
    if (P < 1 || prm->swap_every < 1 || t0 < 0 || rho0 < 0 || rho1 > R) return -1;
    for (int32_t p = 0; p + 1 < P; p++)
        if (!(prm->betas[p] > prm->betas[p + 1])) return -1;
    for (int32_t t = t0; t < t1; t++) {
        for (int32_t chi = 0; chi < pb->n_colours; chi++)
            for (int32_t site = 0; site < n; site++) {
                if (!pb->used[site] || pb->colour[site] != chi) continue;
                for (int32_t p = 0; p < P; p++) {
                    int8_t *slot = s + (int64_t)p * n * R;
                    for (int32_t rho = rho0; rho < rho1; rho++) {
                        int32_t sig = *at(s, n, R, p, site, rho);
                        int32_t delta = (int32_t)orc_flip_delta(pb, slot, R, rho, site);
                        double x = prm->betas[p] * (double)delta;
                        uint32_t u = orc_sweep_uniform(prm->seed, (uint32_t)t,
                                                       (uint32_t)(site * P + p), (uint32_t)rho,
                                                       (uint32_t)inst);
                        if (x <= 0.0 || u < orc_threshold(x)) *at(s, n, R, p, site, rho) = (int8_t)-sig;
                    }
                }
            }
        if ((t + 1) % prm->swap_every == 0 && P > 1) {
            int32_t e = (t + 1) / prm->swap_every - 1;
            pt_energies(pb, s, P, R, rho0, rho1, E);
            for (int32_t p = e & 1; p + 1 < P; p += 2)
                for (int32_t rho = rho0; rho < rho1; rho++) {
                    int64_t dE = E[(int64_t)(p + 1) * R + rho] - E[(int64_t)p * R + rho];
                    int accept = dE <= 0;
                    if (!accept) {
                        uint32_t u = orc_swap_uniform(prm->seed, (uint32_t)e, (uint32_t)p,
                                                      (uint32_t)rho, (uint32_t)inst);
                        accept = u < orc_swap_threshold(prm->betas[p], prm->betas[p + 1], dE);
                    }
                    if (accept) {
                        for (int32_t site = 0; site < n; site++) {
                            int8_t a = *at(s, n, R, p, site, rho);
                            *at(s, n, R, p, site, rho) = *at(s, n, R, p + 1, site, rho);
                            *at(s, n, R, p + 1, site, rho) = a;
                        }
                        int64_t tmp = E[(int64_t)p * R + rho];
                        E[(int64_t)p * R + rho] = E[(int64_t)(p + 1) * R + rho];
                        E[(int64_t)(p + 1) * R + rho] = tmp;
                    }
                }
        }
    }
    pt_energies(pb, s, P, R, rho0, rho1, E);
    return 0;
}
