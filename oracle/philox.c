/*
 * Philox4x32-10, restated from its published definition (Salmon, Moraes, Dror
 * and Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11, Sec. 4.2):
 * ten rounds of two 32x32->64 multiplies with the multipliers 0xD2511F53 and
 * 0xCD9E8D57, the key bumped by the Weyl constants 0x9E3779B9 / 0xBB67AE85
 * between rounds.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 */
#include "oracle.h"

static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    uint32_t n3 = lo0;
    c[0] = n0;
    c[1] = n1;
    c[2] = n2;
    c[3] = n3;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k[0] += 0x9E3779B9u;
            k[1] += 0xBB67AE85u;
        }
        philox_round(c, k);
    }
    for (int i = 0; i < 4; i++) out[i] = c[i];
}

/* Key of a stream: (seed_lo, seed_hi ^ domain). */
static void stream_key(uint64_t seed, uint32_t domain, uint32_t key[2])
{
    key[0] = (uint32_t)seed;
    key[1] = (uint32_t)(seed >> 32) ^ domain;
}

/* The per-attempt uniform of the single-spin sweep (SQA and PT), u = h * 2^25 + l:
 *   h, its 7 high bits: the low 7 bits of byte (r / 8) of output word (r % 4)
 *     of the SWEEP_HI block at counter (t, slot, 2 * (rho / 32) + (r / 4) % 2, inst),
 *     r = rho % 32 (one block serves 16 replicas of a 32-replica word);
 *   l, its 25 low bits: output word (rho % 4) of the SWEEP_LO block at counter
 *     (t, slot, rho / 4, inst), shifted right by 7.
 * Both are independent uniform bit strings, so u is uniform on [0, 2^32). */
uint32_t orc_sweep_uniform(uint64_t seed, uint32_t t, uint32_t slot, uint32_t rho, uint32_t inst)
{
    uint32_t r = rho & 31u;
    uint32_t khi[2], klo[2], a[4], b[4];
    stream_key(seed, ORC_DOM_SWEEP_HI, khi);
    stream_key(seed, ORC_DOM_SWEEP_LO, klo);
    uint32_t ca[4] = {t, slot, 2u * (rho >> 5) + ((r >> 2) & 1u), inst};
    uint32_t cb[4] = {t, slot, rho >> 2, inst};
    orc_philox4x32_10(ca, khi, a);
    orc_philox4x32_10(cb, klo, b);
    uint32_t h = (a[r & 3u] >> (8u * (r >> 3))) & 0x7Fu;
    uint32_t l = b[rho & 3u] >> 7;
    return (h << 25) | l;
}

uint32_t orc_swap_uniform(uint64_t seed, uint32_t event, uint32_t pair, uint32_t rho, uint32_t inst)
{
    uint32_t ctr[4] = {event, pair, rho >> 2, inst};
    uint32_t key[2], out[4];
    stream_key(seed, ORC_DOM_SWAP, key);
    orc_philox4x32_10(ctr, key, out);
    return out[rho & 3u];
}

uint32_t orc_wolff_start(uint64_t seed, uint32_t t, uint32_t site, uint32_t rho, uint32_t inst, int32_t L)
{
    uint32_t ctr[4] = {t, site, rho >> 2, inst};
    uint32_t key[2], out[4];
    stream_key(seed, ORC_DOM_WSTART, key);
    orc_philox4x32_10(ctr, key, out);
    return (uint32_t)(((uint64_t)out[rho & 3u] * (uint64_t)L) >> 32);
}

uint32_t orc_wolff_bond_uniform(uint64_t seed, uint32_t t, uint32_t site, int32_t L, int32_t tau, uint32_t rho,
                                uint32_t inst)
{
    uint32_t key[2], out[4], u = 0;
    stream_key(seed, ORC_DOM_WBOND, key);
    for (uint32_t k = 0; k < 32; k++) {
        uint32_t ctr[4] = {t, site * (uint32_t)L + (uint32_t)tau, (rho >> 5) * 8u + (k >> 2), inst};
        orc_philox4x32_10(ctr, key, out);
        u |= ((out[k & 3u] >> (rho & 31u)) & 1u) << (31u - k);
    }
    return u;
}

uint32_t orc_wolff_accept_uniform(uint64_t seed, uint32_t t, uint32_t site, uint32_t rho, uint32_t inst)
{
    uint32_t ctr[4] = {t, site, rho >> 2, inst};
    uint32_t key[2], out[4];
    stream_key(seed, ORC_DOM_WACC, key);
    orc_philox4x32_10(ctr, key, out);
    return out[rho & 3u];
}

/* Initial spin of (site, z, replica rho): bit (rho % 32) of output word
 * (rho/32) % 4 of the INIT stream at counter (site, z, rho/128, inst). */
void orc_init_spins(const orc_problem *pb, int32_t Z, int32_t R, uint64_t seed, int32_t inst,
                    int8_t *s)
{
    uint32_t key[2];
    stream_key(seed, ORC_DOM_INIT, key);
    for (int32_t z = 0; z < Z; z++)
        for (int32_t site = 0; site < pb->n; site++)
            for (int32_t rho = 0; rho < R; rho++) {
                int8_t v = 1;
                if (pb->used[site]) {
                    uint32_t w = (uint32_t)rho >> 5;
                    uint32_t ctr[4] = {(uint32_t)site, (uint32_t)z, w >> 2, (uint32_t)inst};
                    uint32_t out[4];
                    orc_philox4x32_10(ctr, key, out);
                    uint32_t bit = (out[w & 3u] >> ((uint32_t)rho & 31u)) & 1u;
                    v = bit ? -1 : 1;
                }
                s[((int64_t)z * pb->n + site) * R + rho] = v;
            }
}

/* Uniform labelled tree (Pruefer sequence) element: floor(u * N / 2^32). */
uint32_t orc_tree_draw(uint64_t seed, int32_t inst, int32_t tree, int32_t pos, int32_t N)
{
    uint32_t key[2], out[4];
    uint32_t ctr[4] = {(uint32_t)tree, (uint32_t)pos, 0u, (uint32_t)inst};
    stream_key(seed, ORC_DOM_TREE, key);
    orc_philox4x32_10(ctr, key, out);
    return (uint32_t)(((uint64_t)out[0] * (uint64_t)N) >> 32);
}
