/*
 * oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU restatement of the checkerboard
 * Metropolis / facilitated sweep of Levy, Cohen & Rabani, "Simulating
 * lattice spin models on GPUs" (arXiv:1209.0296).  It exists to check the
 * CUDA library against the paper; nothing in the product path may call it.
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * reference legs load this file's shared object.
 *
 * It shares no code, header, table or constant generator with the CUDA
 * library: Philox4x32-10, the acceptance rule, the initial state and the
 * observables are all written out again here, site by site, in the order
 * the paper's algorithm states them.
 *
 * Readings of the paper taken here (the paper is silent or ambiguous):
 *  - Hamiltonian sign: H = -J sum_<ij> s_i s_j - h sum_i s_i for every model
 *    (Eq. 2 sign, extended with a field); the North-East model of Eq. 3
 *    with B = +1 is h = -1 here.  Each bond (i, i+e_d) is counted once per
 *    direction d, so for L = 2 a pair appears twice, in H and in dE alike.
 *  - Checkerboard: colour(x,y[,z]) = (x+y[+z]) mod 2; one sweep updates
 *    colour 0 then colour 1 (the paper's red+blue, then green+white, §III.A
 *    steps 6-7 and Fig. 2).  Periodic boundaries; L even.
 *  - Randomness: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) in place
 *    of the paper's per-thread LCG (§IV, Eqs. 5-7).  key = (seed lo, seed
 *    hi); counter = (g, sweep lo, sweep hi, colour); g = r*G + (j >> sh),
 *    r = y + L*z the row, j = x >> 1 the index of the site among the
 *    same-colour sites of its row, G = ceil((L/2) / 2^sh) groups per row,
 *    sh = 2 for spin-1/2 (word j & 3 decides acceptance), sh = 1 for
 *    spin-S > 1/2 (word 2(j&1) decides acceptance, word 2(j&1)+1 picks the
 *    proposal).  Initial states use counter (i >> 2, 0, 0, 2), word i & 3.
 *  - Acceptance (§III.A, min[1, exp(-dH/T)]): dE <= 0 accepts without a
 *    draw; otherwise accept iff u < floor(exp(-dE/T) * 2^32).
 *  - Spin-S (§III "any spin value"): state k in [0, two_S]; s = 2k - two_S
 *    for odd two_S, s = k - two_S/2 for even two_S.  Proposal: one of the
 *    other two_S states, uniformly: k' = (k + 1 + floor(u*two_S/2^32)) mod
 *    (two_S + 1).
 *  - North-East (§III.B): north of (x,y) is (x, y-1), east is (x+1, y); a
 *    site may change only if both are up (+1).  With J = h = 0 the last
 *    model parameter is the up-spin concentration c and the rates are
 *    p(down->up) = min(1, c/(1-c)), p(up->down) = min(1, (1-c)/c).
 *  - Persistence: a site's flag is set the first time its value changes
 *    (North-East model only).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, as published by Salmon et al. (SC'11, "Parallel random     */
/* numbers: as easy as 1, 2, 3"): ten rounds of two 32x32->64 multiplies     */
/* with the round keys bumped by the Weyl constants between rounds.         */
/* ------------------------------------------------------------------------ */
void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                          uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* One Philox draw for (seed, counter words). */
static uint32_t draw_word(uint64_t seed, uint32_t g, int64_t sweep,
                          uint32_t colour, int word)
{
    uint32_t ctr[4] = {g, (uint32_t)((uint64_t)sweep & 0xffffffffu),
                       (uint32_t)((uint64_t)sweep >> 32), colour};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t out[4];
    oracle_philox4x32_10(ctr, key, out);
    return out[word];
}

/* ------------------------------------------------------------------------ */
/* Spin values (§III: s_i = +-1, "easily extended to any spin value").      */
/* ------------------------------------------------------------------------ */
int oracle_spin_of_state(int two_S, int k)
{
    if (two_S & 1) return 2 * k - two_S;
    return k - two_S / 2;
}

int oracle_state_of_spin(int two_S, int s)
{
    if (two_S & 1) return (s + two_S) / 2;
    return s + two_S / 2;
}

/* ------------------------------------------------------------------------ */
/* Metropolis acceptance threshold (§III.A: P_acc = min[1, exp(-dH/T)]).    */
/* Returns 1 when the move is accepted without a draw (dE <= 0); otherwise  */
/* returns 0 and writes thr = floor(exp(-dE/T) * 2^32), so that a uniform   */
/* 32-bit draw u accepts with probability exactly thr / 2^32.               */
/* ------------------------------------------------------------------------ */
int oracle_metropolis_threshold(double dE, double T, uint32_t *thr)
{
    if (dE <= 0.0) {
        *thr = 0;
        return 1;
    }
    double p = exp(-dE / T);
    *thr = (uint32_t)floor(ldexp(p, 32));
    return 0;
}

/* Same rule when the acceptance probability p itself is given (North-East
 * model at fixed concentration c, §III.B). */
int oracle_probability_threshold(double p, uint32_t *thr)
{
    if (p >= 1.0) {
        *thr = 0;
        return 1;
    }
    *thr = (uint32_t)floor(ldexp(p, 32));
    return 0;
}

/* Energy change of replacing spin s by s2 at a site whose neighbour spins
 * sum to n, for H = -J sum s_i s_j - h sum s_i (Eq. 2 plus a field). */
double oracle_delta_energy(double J, double h, int ds, int n)
{
    return -(J * (double)(ds * n)) - h * (double)ds;
}

/* ------------------------------------------------------------------------ */
/* Lattice geometry.                                                         */
/* ------------------------------------------------------------------------ */
typedef struct {
    int dims, L, two_S, model;
    double J, h, T, c;
    int cmode;
    uint64_t seed;
    int64_t N;
    const int8_t *eps;   /* per-bond signs (Eq. 1's J_ij / J), or NULL: all +1 */
    const int8_t *eta;   /* per-site field signs (Eq. 1's B_i / h), or NULL: all +1 */
} params_t;

static int64_t site_index(const params_t *p, int x, int y, int z)
{
    int L = p->L;
    x = ((x % L) + L) % L;
    y = ((y % L) + L) % L;
    z = ((z % L) + L) % L;
    return (int64_t)x + (int64_t)L * ((int64_t)y + (int64_t)L * (int64_t)z);
}

static int setup(params_t *p, int dims, int L, int two_S, int model, double J,
                 double h, double T_or_c, uint64_t seed)
{
    if (dims != 2 && dims != 3) return -1;
    if (L < 2 || (L & 1)) return -1;
    if (two_S < 1 || two_S > 8) return -1;
    if (model != 0 && model != 1 && model != 2) return -1;
    if (model == 1 && (dims != 2 || two_S != 1)) return -1;
    p->eps = NULL;
    p->eta = NULL;
    p->dims = dims; p->L = L; p->two_S = two_S; p->model = model;
    p->J = J; p->h = h; p->seed = seed;
    p->N = (int64_t)L * L * (dims == 3 ? L : 1);
    if (p->N >= ((int64_t)1 << 32)) return -1;
    p->cmode = (model == 1 && J == 0.0 && h == 0.0);
    if (p->cmode) {
        if (!(T_or_c > 0.0 && T_or_c < 1.0)) return -1;
        p->c = T_or_c; p->T = 0.0;
    } else {
        if (!(T_or_c > 0.0)) return -1;
        p->T = T_or_c; p->c = 0.0;
    }
    return 0;
}

/* Sign of the bond from site (x,y,z) to its +e_d neighbour: eps[d*N + i]  */
/* with i the linear index of (x,y,z) (Eq. 1 with J_ij = J * eps), or +1.   */
static int bond_sign(const params_t *p, int x, int y, int z, int d)
{
    if (p->eps == NULL) return 1;
    return p->eps[(int64_t)d * p->N + site_index(p, x, y, z)];
}

/* Sum over the 2*dims nearest neighbours j of (x,y,z) of eps_ij * s_j,      */
/* periodic (with no couplings set: the plain neighbour sum).               */
static int neighbour_sum(const params_t *p, const int8_t *s, int x, int y,
                         int z)
{
    int n = bond_sign(p, x - 1, y, z, 0) * s[site_index(p, x - 1, y, z)] +
            bond_sign(p, x, y, z, 0) * s[site_index(p, x + 1, y, z)] +
            bond_sign(p, x, y - 1, z, 1) * s[site_index(p, x, y - 1, z)] +
            bond_sign(p, x, y, z, 1) * s[site_index(p, x, y + 1, z)];
    if (p->dims == 3)
        n += bond_sign(p, x, y, z - 1, 2) * s[site_index(p, x, y, z - 1)] +
             bond_sign(p, x, y, z, 2) * s[site_index(p, x, y, z + 1)];
    return n;
}

/* ------------------------------------------------------------------------ */
/* Initial state (§III.A step 1: random lattice; §III.B step 1: each site up */
/* with probability c).  init: 0 cold (+1 / top state), 1 random, 2          */
/* equilibrium at concentration c (North-East, c-mode).                      */
/* ------------------------------------------------------------------------ */
int oracle_init(int dims, int L, int two_S, int model, double J, double h,
                double T_or_c, uint64_t seed, int init, int8_t *s)
{
    params_t p;
    if (setup(&p, dims, L, two_S, model, J, h, T_or_c, seed)) return -1;
    if (init == 2 && !p.cmode) return -1;
    for (int64_t i = 0; i < p.N; ++i) {
        uint32_t u = draw_word(seed, (uint32_t)(i >> 2), 0, 2, (int)(i & 3));
        int k;
        if (model == 2) {                              /* Potts: the state label */
            if (init == 0) k = 0;
            else if (init == 1)
                k = (two_S == 1) ? ((u < 0x80000000u) ? 0 : 1)
                                 : (int)(((uint64_t)u * (uint64_t)(two_S + 1)) >> 32);
            else return -1;
            s[i] = (int8_t)k;
            continue;
        }
        if (init == 0) {
            k = two_S;                                 /* all spins up */
        } else if (init == 1) {
            if (two_S == 1) k = (u < 0x80000000u) ? 1 : 0;
            else k = (int)(((uint64_t)u * (uint64_t)(two_S + 1)) >> 32);
        } else if (init == 2) {
            uint32_t thr_c = (uint32_t)floor(ldexp(p.c, 32));
            k = (u < thr_c) ? 1 : 0;
        } else {
            return -1;
        }
        s[i] = (int8_t)oracle_spin_of_state(two_S, k);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Observables of one configuration, straight from their definitions:        */
/*   bond = sum over sites i and directions d of s_i * s_{i+e_d}             */
/*   mag  = sum_i s_i;  up = #{s_i > 0};  unflipped = #{flag_i == 0}         */
/* E = -J*bond - h*mag (Eq. 2 with a field).                                 */
/* ------------------------------------------------------------------------ */
void oracle_measure_couplings(int dims, int L, const int8_t *s, const uint8_t *flag,
                              const int8_t *eps, int64_t *bond, int64_t *mag,
                              int64_t *up, int64_t *unflipped);

/* With couplings (eps != NULL) the bond sum is weighted:                    */
/*   bond = sum over sites i and directions d of eps_{i,d} s_i s_{i+e_d};    */
/* with field signs eta (may be NULL) field = sum_i eta_i s_i, so that       */
/* E = -J*bond - h*field (Eq. 1 with J_ij = J eps_ij, B_i = h eta_i).        */
void oracle_measure_disorder(int dims, int L, const int8_t *s, const uint8_t *flag,
                             const int8_t *eps, const int8_t *eta, int64_t *bond,
                             int64_t *mag, int64_t *up, int64_t *unflipped,
                             int64_t *field)
{
    int64_t fs = 0;
    const int64_t N = (int64_t)L * L * (dims == 3 ? L : 1);
    for (int64_t i = 0; i < N; ++i) fs += (eta == NULL ? 1 : eta[i]) * (int64_t)s[i];
    if (field) *field = fs;
    oracle_measure_couplings(dims, L, s, flag, eps, bond, mag, up, unflipped);
}

void oracle_measure_couplings(int dims, int L, const int8_t *s, const uint8_t *flag,
                              const int8_t *eps, int64_t *bond, int64_t *mag,
                              int64_t *up, int64_t *unflipped)
{
    params_t p;
    memset(&p, 0, sizeof p);
    p.dims = dims; p.L = L;
    p.N = (int64_t)L * L * (dims == 3 ? L : 1);
    p.eps = eps;
    int Lz = (dims == 3) ? L : 1;
    int64_t b = 0, m = 0, nu = 0, nf = 0;
    for (int z = 0; z < Lz; ++z)
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                int64_t i = site_index(&p, x, y, z);
                int si = s[i];
                b += bond_sign(&p, x, y, z, 0) * si * s[site_index(&p, x + 1, y, z)];
                b += bond_sign(&p, x, y, z, 1) * si * s[site_index(&p, x, y + 1, z)];
                if (dims == 3) b += bond_sign(&p, x, y, z, 2) * si * s[site_index(&p, x, y, z + 1)];
                m += si;
                nu += (si > 0);
                nf += (flag == NULL) ? 0 : (flag[i] == 0);
            }
    *bond = b; *mag = m; *up = nu; *unflipped = nf;
}

/* Potts observables (q states, labels 0..q-1):                             */
/*   bond = number of bonds (i, i+e_d) with equal ends, mag = number of      */
/*   sites in state 0, up = number of sites in another state; so that        */
/*   E = -J*bond - h*mag for H = -J sum delta(s_i,s_j) - h sum delta(s_i,0). */
void oracle_measure_potts(int dims, int L, const int8_t *s, int64_t *bond,
                          int64_t *mag, int64_t *up)
{
    params_t p;
    memset(&p, 0, sizeof p);
    p.dims = dims; p.L = L;
    int Lz = (dims == 3) ? L : 1;
    int64_t b = 0, m = 0, nu = 0;
    for (int z = 0; z < Lz; ++z)
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                int si = s[site_index(&p, x, y, z)];
                b += (si == s[site_index(&p, x + 1, y, z)]);
                b += (si == s[site_index(&p, x, y + 1, z)]);
                if (dims == 3) b += (si == s[site_index(&p, x, y, z + 1)]);
                m += (si == 0);
                nu += (si != 0);
            }
    *bond = b; *mag = m; *up = nu;
}

void oracle_measure(int dims, int L, const int8_t *s, const uint8_t *flag,
                    int64_t *bond, int64_t *mag, int64_t *up,
                    int64_t *unflipped)
{
    oracle_measure_couplings(dims, L, s, flag, NULL, bond, mag, up, unflipped);
}

/* ------------------------------------------------------------------------ */
/* The sweep (§III.A algorithm steps 5-8, Fig. 2; §III.B facilitated rule,   */
/* Eq. 3).  For each sweep t: all colour-0 sites, then all colour-1 sites;   */
/* sites of one colour share no bond and no north/east neighbour, so the     */
/* order inside a colour does not matter and a plain raster loop is used.    */
/* After each sweep the four observables are recorded (NULL skips one).     */
/* flag may be NULL for the Ising model.                                     */
/* ------------------------------------------------------------------------ */
/* eps: per-bond signs (Eq. 1 with J_ij = J * eps_ij, nearest neighbours),  */
/* eps[d*N + i] for the bond from linear site i to its +e_d neighbour; NULL */
/* for uniform couplings.  Ising model only.                                */
/* eta: per-site field signs (B_i = h * eta_i), or NULL for a uniform field; */
/* field[k] (may be NULL) receives sum_i eta_i s_i after each sweep.         */
int oracle_sweep_disorder(int dims, int L, int two_S, int model, double J, double h,
                          double T_or_c, uint64_t seed, int8_t *s, uint8_t *flag,
                          const int8_t *eps, const int8_t *eta, int64_t sweep0,
                          int64_t nsweeps, int64_t *bond, int64_t *mag, int64_t *up,
                          int64_t *unflipped, int64_t *field)
{
    params_t p;
    if (setup(&p, dims, L, two_S, model, J, h, T_or_c, seed)) return -1;
    if ((eps != NULL || eta != NULL) && model != 0) return -1;
    p.eps = eps;
    p.eta = eta;
    if (model == 1 && flag == NULL) return -1;
    const int sh = (two_S == 1) ? 2 : 1;               /* sites per draw: 4 or 2 */
    const int64_t half = L / 2;
    const int64_t G = (half + (1 << sh) - 1) >> sh;    /* groups per row */
    const int Lz = (dims == 3) ? L : 1;

    for (int64_t t = sweep0; t < sweep0 + nsweeps; ++t) {
        for (int colour = 0; colour < 2; ++colour) {
            for (int z = 0; z < Lz; ++z)
                for (int y = 0; y < L; ++y)
                    for (int x = 0; x < L; ++x) {
                        if (((x + y + z) & 1) != colour) continue;
                        int64_t i = site_index(&p, x, y, z);
                        int64_t r = (int64_t)y + (int64_t)L * z;
                        int64_t j = x >> 1;
                        uint32_t g = (uint32_t)(r * G + (j >> sh));

                        int s_old = s[i];
                        int k_old = (model == 2) ? s_old : oracle_state_of_spin(two_S, s_old);
                        int k_new;
                        uint32_t u_acc;
                        if (two_S == 1) {
                            k_new = 1 - k_old;                 /* spin flip */
                            u_acc = draw_word(seed, g, t, (uint32_t)colour,
                                              (int)(j & 3));
                        } else {
                            int w = 2 * (int)(j & 1);
                            u_acc = draw_word(seed, g, t, (uint32_t)colour, w);
                            uint32_t u_prop = draw_word(seed, g, t,
                                                        (uint32_t)colour, w + 1);
                            int step = 1 + (int)(((uint64_t)u_prop *
                                                  (uint64_t)two_S) >> 32);
                            k_new = (k_old + step) % (two_S + 1);
                        }
                        int s_new = (model == 2) ? k_new : oracle_spin_of_state(two_S, k_new);

                        /* Potts (q = two_S + 1 states): H = -J sum delta(s_i,s_j)
                         * - h sum delta(s_i,0); the move changes the number of
                         * equal neighbours by dn and the state-0 count by df. */
                        if (model == 2) {
                            int dn = 0;
                            const int nb[6] = {
                                s[site_index(&p, x - 1, y, z)], s[site_index(&p, x + 1, y, z)],
                                s[site_index(&p, x, y - 1, z)], s[site_index(&p, x, y + 1, z)],
                                dims == 3 ? s[site_index(&p, x, y, z - 1)] : 0,
                                dims == 3 ? s[site_index(&p, x, y, z + 1)] : 0};
                            for (int d = 0; d < 2 * dims; ++d) dn += (nb[d] == s_new) - (nb[d] == s_old);
                            const int df = (s_new == 0) - (s_old == 0);
                            const double dE = -(J * (double)dn) - h * (double)df;
                            uint32_t thr;
                            int accept = oracle_metropolis_threshold(dE, p.T, &thr);
                            if (!accept) accept = (u_acc < thr);
                            if (accept) s[i] = (int8_t)s_new;
                            continue;
                        }

                        /* North-East constraint (§III.B): both the north
                         * (x, y-1) and the east (x+1, y) neighbours up. */
                        if (model == 1) {
                            int north = s[site_index(&p, x, y - 1, z)];
                            int east = s[site_index(&p, x + 1, y, z)];
                            if (!(north == 1 && east == 1)) continue;
                        }

                        int accept;
                        uint32_t thr;
                        if (model == 1 && p.cmode) {
                            double pr = (s_new > s_old) ? p.c / (1.0 - p.c)
                                                        : (1.0 - p.c) / p.c;
                            accept = oracle_probability_threshold(pr, &thr);
                        } else {
                            int n = neighbour_sum(&p, s, x, y, z);
                            const double hi = (eta == NULL || eta[i] > 0) ? h : -h;   /* B_i */
                            double dE = oracle_delta_energy(J, hi, s_new - s_old, n);
                            accept = oracle_metropolis_threshold(dE, p.T, &thr);
                        }
                        if (!accept) accept = (u_acc < thr);
                        if (accept) {
                            s[i] = (int8_t)s_new;
                            if (flag != NULL && s_new != s_old) flag[i] = 1;
                        }
                    }
        }
        int64_t b, m, nu, nf = 0, fs = 0;
        if (model == 2) oracle_measure_potts(dims, L, s, &b, &m, &nu);
        else oracle_measure_disorder(dims, L, s, flag, eps, eta, &b, &m, &nu, &nf, &fs);
        if (field) field[t - sweep0] = fs;
        int64_t k = t - sweep0;
        if (bond) bond[k] = b;
        if (mag) mag[k] = m;
        if (up) up[k] = nu;
        if (unflipped) unflipped[k] = nf;
    }
    return 0;
}

int oracle_sweep_couplings(int dims, int L, int two_S, int model, double J, double h,
                           double T_or_c, uint64_t seed, int8_t *s, uint8_t *flag,
                           const int8_t *eps, int64_t sweep0, int64_t nsweeps,
                           int64_t *bond, int64_t *mag, int64_t *up,
                           int64_t *unflipped)
{
    return oracle_sweep_disorder(dims, L, two_S, model, J, h, T_or_c, seed, s, flag, eps, NULL,
                                 sweep0, nsweeps, bond, mag, up, unflipped, NULL);
}

int oracle_sweep(int dims, int L, int two_S, int model, double J, double h,
                 double T_or_c, uint64_t seed, int8_t *s, uint8_t *flag,
                 int64_t sweep0, int64_t nsweeps, int64_t *bond,
                 int64_t *mag, int64_t *up, int64_t *unflipped)
{
    return oracle_sweep_couplings(dims, L, two_S, model, J, h, T_or_c, seed, s, flag, NULL,
                                  sweep0, nsweeps, bond, mag, up, unflipped);
}

/* ------------------------------------------------------------------------ */
/* The paper's own North-East GPU algorithm (§III.B, the second algorithm:   */
/* steps 3-10, Figs. 4-5): random sub-lattices and random sites instead of   */
/* a checkerboard, to keep the serial relaxation dynamics.  2D spin-1/2.     */
/*                                                                           */
/* The lattice is cut into Q = (L/b)^2 square sub-lattices of P = b*b spins  */
/* (step 3).  One sweep is two launches (steps 9-10); in each launch every   */
/* sub-lattice (step 5: each is picked by exactly one block) makes q rounds  */
/* of lambda concurrent random picks with q * lambda = P/2 (steps 6-8).      */
/* Sites outside a sub-lattice (its boundary, step 5) keep the values they   */
/* had when the launch started.                                              */
/*                                                                           */
/* Readings taken here (the paper leaves them open):                         */
/*  - Thread i of sub-lattice B (row-major over sub-lattices) makes one     */
/*    Philox call per two rounds: in launch l of sweep t, rounds 2k and 2k+1 */
/*    share the call with counter (B*C + k*lambda + i, t lo, t hi, 4 + l),   */
/*    C = ceil(q/2)*lambda calls per sub-lattice; round r uses words         */
/*    w = 2*(r & 1) (the site, floor(w * P / 2^32) row-major inside the      */
/*    sub-lattice) and w + 1 (the acceptance draw).  The block-to-           */
/*    sub-lattice permutation of step 5 changes nothing (every sub-lattice  */
/*    is processed once per launch, blocks do not interact within one) and  */
/*    is the identity.                                                       */
/*  - The lambda picks of a round are concurrent: each is decided from the   */
/*    state at the start of the round; when several pick the same site, the  */
/*    lowest thread index's outcome is kept.                                 */
/*  - A neighbour inside the sub-lattice is read live; one outside it from   */
/*    the launch's frozen input.  With one sub-lattice (b = L) every        */
/*    neighbour is inside, so Q = lambda = 1 is serial random-site           */
/*    Metropolis, the paper's reference limit.                               */
/*  - Move rule and thresholds as in oracle_sweep: flip, the North-East      */
/*    constraint, accept without a draw when allowed by "always", else iff   */
/*    u < thr.  Persistence flags as in oracle_sweep.                        */
/*                                                                           */
/* The balance-preserving variant (§III.B, after Fig. 5: steps 6-9 changed) */
/* picks the lambda sites of a round among one colour only, red and white   */
/* rounds alternating, and takes four launches per sweep.  Its round count  */
/* per launch is not legible in the paper; read here as q/2 (so a sweep     */
/* still makes q*lambda*2 = P picks per sub-lattice, the time unit of the   */
/* serial reference), which needs q/2 even.  Red is colour 0, (x+y) even,  */
/* and goes first; a round of colour c uses the same Philox words as round */
/* r of the plain algorithm, with the site word mapped into the P/2 sites  */
/* of that colour: m = floor(w * P/2 / 2^32), row ly = m / (b/2), column   */
/* lx = 2 (m mod b/2) + ((ly + c) & 1).  Launches 0..3 use tags 4..7.     */
/* With one sub-lattice a round changes only non-interacting sites, each by */
/* a Metropolis move, so the Boltzmann distribution is stationary for any  */
/* lambda -- the paper's point for this variant.                            */
/* ------------------------------------------------------------------------ */
static int rsite_accept(const params_t *p, int model, int s_old, int s_new, int n, uint32_t u)
{
    uint32_t thr;
    int accept;
    if (model == 1 && p->cmode) {
        double pr = (s_new > s_old) ? p->c / (1.0 - p->c) : (1.0 - p->c) / p->c;
        accept = oracle_probability_threshold(pr, &thr);
    } else {
        double dE = oracle_delta_energy(p->J, p->h, s_new - s_old, n);
        accept = oracle_metropolis_threshold(dE, p->T, &thr);
    }
    if (!accept) accept = (u < thr);
    return accept;
}

/* balanced = 0: the algorithm of steps 3-10; 1: the balance-preserving    */
/* variant described above.                                                  */
int oracle_rsite_sweep_variant(int L, int model, double J, double h, double T_or_c,
                               uint64_t seed, int b, int lambda, int balanced, int8_t *s,
                               uint8_t *flag, int64_t sweep0, int64_t nsweeps, int64_t *bond,
                               int64_t *mag, int64_t *up, int64_t *unflipped)
{
    params_t p;
    if (setup(&p, 2, L, 1, model, J, h, T_or_c, seed)) return -1;
    if (model == 1 && flag == NULL) return -1;
    if (b < 2 || (b & (b - 1)) != 0 || L % b != 0) return -1;
    const int64_t P = (int64_t)b * b;
    if (lambda < 1 || (P / 2) % lambda != 0) return -1;
    const int64_t q = P / 2 / lambda;
    if (balanced && (q % 4) != 0) return -1;
    const int launches = balanced ? 4 : 2;
    const int64_t rounds = balanced ? q / 2 : q;        /* rounds per launch */
    const int64_t calls = (rounds + 1) / 2 * lambda;   /* Philox calls per sub-lattice and launch */
    const int nt = L / b;
    int8_t *src = (int8_t *)malloc((size_t)p.N);
    int8_t *loc = (int8_t *)malloc((size_t)P);
    int8_t *nv = (int8_t *)malloc((size_t)lambda);
    int64_t *pick = (int64_t *)malloc(sizeof(int64_t) * (size_t)lambda);
    if (!src || !loc || !nv || !pick) {
        free(src); free(loc); free(nv); free(pick);
        return -1;
    }
    const uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    for (int64_t t = sweep0; t < sweep0 + nsweeps; ++t) {
        for (int launch = 0; launch < launches; ++launch) {
            memcpy(src, s, (size_t)p.N);               /* the launch's input */
            for (int ty = 0; ty < nt; ++ty)
                for (int tx = 0; tx < nt; ++tx) {
                    const int64_t B = (int64_t)ty * nt + tx;
                    const int x0 = tx * b, y0 = ty * b;
                    for (int ly = 0; ly < b; ++ly)
                        for (int lx = 0; lx < b; ++lx)
                            loc[ly * b + lx] = src[site_index(&p, x0 + lx, y0 + ly, 0)];
                    for (int64_t r = 0; r < rounds; ++r) {
                        /* every pick of the round decided from the same state */
                        for (int i = 0; i < lambda; ++i) {
                            uint32_t ctr[4] = {(uint32_t)(B * calls + (r / 2) * lambda + i),
                                               (uint32_t)((uint64_t)t & 0xffffffffu),
                                               (uint32_t)((uint64_t)t >> 32),
                                               (uint32_t)(4 + launch)};
                            uint32_t w[4];
                            oracle_philox4x32_10(ctr, key, w);
                            const int ws = 2 * (int)(r & 1);
                            int64_t site;
                            if (!balanced) {
                                site = (int64_t)(((uint64_t)w[ws] * (uint64_t)P) >> 32);
                            } else {            /* round colour c = r & 1 */
                                const int64_t m = (int64_t)(((uint64_t)w[ws] * (uint64_t)(P / 2)) >> 32);
                                const int64_t row = m / (b / 2);
                                site = row * b + 2 * (m % (b / 2)) + ((row + (r & 1)) & 1);
                            }
                            const int lx = (int)(site % b), ly = (int)(site / b);
                            int nb[4];   /* north, east, south, west */
                            const int dx[4] = {0, 1, 0, -1}, dy[4] = {-1, 0, 1, 0};
                            for (int d = 0; d < 4; ++d) {
                                const int X = ((x0 + lx + dx[d]) % L + L) % L;
                                const int Y = ((y0 + ly + dy[d]) % L + L) % L;
                                if (X >= x0 && X < x0 + b && Y >= y0 && Y < y0 + b)
                                    nb[d] = loc[(Y - y0) * b + (X - x0)];
                                else
                                    nb[d] = src[site_index(&p, X, Y, 0)];
                            }
                            const int s_old = loc[site], s_new = -s_old;
                            int allowed = 1;
                            if (model == 1) allowed = (nb[0] == 1 && nb[1] == 1);
                            const int n = nb[0] + nb[1] + nb[2] + nb[3];
                            nv[i] = (int8_t)((allowed && rsite_accept(&p, model, s_old, s_new, n, w[ws + 1]))
                                                 ? s_new : s_old);
                            pick[i] = site;
                        }
                        /* apply: the first pick of a site wins */
                        for (int i = 0; i < lambda; ++i) {
                            int first = 1;
                            for (int j = 0; j < i; ++j)
                                if (pick[j] == pick[i]) first = 0;
                            if (!first) continue;
                            if (nv[i] != loc[pick[i]]) {
                                loc[pick[i]] = nv[i];
                                if (flag != NULL) {
                                    const int lx = (int)(pick[i] % b), ly = (int)(pick[i] / b);
                                    flag[site_index(&p, x0 + lx, y0 + ly, 0)] = 1;
                                }
                            }
                        }
                    }
                    for (int ly = 0; ly < b; ++ly)
                        for (int lx = 0; lx < b; ++lx)
                            s[site_index(&p, x0 + lx, y0 + ly, 0)] = loc[ly * b + lx];
                }
        }
        int64_t bb, m, nu, nf;
        oracle_measure(2, L, s, flag, &bb, &m, &nu, &nf);
        const int64_t k = t - sweep0;
        if (bond) bond[k] = bb;
        if (mag) mag[k] = m;
        if (up) up[k] = nu;
        if (unflipped) unflipped[k] = nf;
    }
    free(src); free(loc); free(nv); free(pick);
    return 0;
}

int oracle_rsite_sweep(int L, int model, double J, double h, double T_or_c,
                       uint64_t seed, int b, int lambda, int8_t *s, uint8_t *flag,
                       int64_t sweep0, int64_t nsweeps, int64_t *bond,
                       int64_t *mag, int64_t *up, int64_t *unflipped)
{
    return oracle_rsite_sweep_variant(L, model, J, h, T_or_c, seed, b, lambda, 0, s, flag, sweep0,
                                      nsweeps, bond, mag, up, unflipped);
}

/* Overlap of a configuration with a reference one, sum_i s_i * ref_i: the  */
/* numerator of the spin-spin autocorrelation Phi(t), §III.B Eq. 4 (the sum */
/* over sites i of s_i(t) s_i(0)).  Both arrays in the same site order.      */
int64_t oracle_overlap(int64_t n, const int8_t *s, const int8_t *ref)
{
    int64_t c = 0;
    for (int64_t i = 0; i < n; ++i) c += (int64_t)s[i] * (int64_t)ref[i];
    return c;
}

/* Potts overlap with a reference configuration: the number of sites whose  */
/* label equals the reference label, sum_i delta(s_i, ref_i).  Eq. 4 is     */
/* written for spins; for labels the product s_i(t) s_i(0) has no meaning,   */
/* and delta(s_i(t), s_i(0)) is the Potts counterpart (for q = 2 with        */
/* sigma = 1 - 2s it is (N + sum_i sigma_i(t) sigma_i(0)) / 2).              */
int64_t oracle_overlap_potts(int64_t n, const int8_t *s, const int8_t *ref)
{
    int64_t c = 0;
    for (int64_t i = 0; i < n; ++i) c += (s[i] == ref[i]) ? 1 : 0;
    return c;
}

/* Number of distinct 32-bit words this oracle needs from Philox per call. */
int oracle_sites_per_draw(int two_S) { return two_S == 1 ? 4 : 2; }
