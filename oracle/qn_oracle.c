/*
 * qn_oracle.c -- plain, slow FP64 CPU oracle for stochastic noisy-QAOA ensembles.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file; only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg
 * (and its reference arm) use it.  It shares no code, header, table or constant
 * generator with the CUDA library: every formula below is written out again from
 * the paper's definitions.
 *
 * What it computes (arXiv 2210.15874, "Stochastic Approach For Simulating
 * Quantum Noise Using Tensor Networks"):
 *
 *   O1  density matrix.  rho <- U rho U^dagger for every gate, then each noise
 *       channel as the operator sum E(rho) = sum_j K_j rho K_j^dagger
 *       (Sec. "Modeling Noise", Eq. op_sum), with the depolarizing Kraus set of
 *       the same section and the textbook amplitude-damping Kraus pair.
 *       sigma_exact = diag(rho)  (Sec. "Stochastic Noise Implementation").
 *
 *   O2  trajectories.  Every gate of the ideal circuit is applied in its
 *       original order; after each gate one uniform number per channel picks a
 *       Kraus operator, whose Pauli (or damping operator) is applied to the
 *       state (Sec. "Stochastic Noise Implementation").  phi = |psi|^2 and
 *       sigma_approx = sum_k phi_k / K (same section).
 *
 * Readings of the paper where it is silent:
 *   - depolarizing parameter: param=0 gives p = total non-identity probability,
 *     each 1q Pauli p/3 (lambda = 4p/3); param=1 takes the paper's lambda,
 *     K0 = sqrt(1-3 lambda/4) I  ->  p = 3 lambda / 4 (1q), 15 lambda / 16 (2q).
 *   - 2q noise: twoq_mode=0 is the 15-Pauli two-qubit depolarizing channel
 *     (each non-II Pauli p/15); twoq_mode=1 is the product of two 1q channels
 *     (Fig. 2's per-qubit noise on a 2q gate).
 *   - Kraus order I, X, Y, Z; 2q code 4a+b, a on the edge's first qubit.
 *     Integer cumulative thresholds T_k = floor(2^32 c_k) in FP64; the first k
 *     with w < T_k is taken, the last bucket takes the rest.
 *   - every gate is noisy (the Hadamard layer included); order per gate:
 *     gate, depolarizing Pauli, damping on the first qubit, damping on the
 *     second qubit.
 *   - QAOA: H on every qubit; per layer l, for every edge (i,j) in list order
 *     diag(1, e^{-i gamma_l}, e^{-i gamma_l}, 1), then for every qubit q = 0..n-1
 *     exp(-i beta_l X) = [[cos b, -i sin b], [-i sin b, cos b]].  Basis index bit
 *     q is qubit q.  C(x) = number of edges (i,j) with x_i != x_j.
 *   - randomness: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with key
 *     (seed_lo, seed_hi) and counter (gate g, 0, t_lo, t_hi) for trajectory t;
 *     word 0 picks the Pauli, words 1 and 2 give the damping draws of the
 *     gate's first and second qubit as u = (w + 0.5) 2^-32.
 *   - damping: p1 = gamma * sum_{x_q=1} |psi_x|^2 / sum_x |psi_x|^2; K1 is taken
 *     when u < p1; the state is renormalised after every damping site.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

enum { ORC_H = 0, ORC_ZZ = 1, ORC_RX = 2 };

typedef struct {
    int32_t kind;   /* ORC_H, ORC_ZZ or ORC_RX */
    int32_t q0, q1; /* q1 = -1 for 1q gates */
    double angle;   /* gamma for ZZ, beta for RX, unused for H */
} orc_gate;

typedef struct {
    double p1, p2, damping;
    int32_t twoq_mode; /* 0: 15-Pauli 2q depolarizing, 1: product of two 1q channels */
    int32_t param;     /* 0: p = total Pauli probability, 1: paper's lambda */
} orc_noise;

/* ------------------------------------------------------------------------- */
/* Philox4x32-10, written from the round description of Salmon et al. (SC'11): */
/* each round multiplies counter words 0 and 2 by two fixed odd constants,     */
/* XORs the high halves with the other two words and the key, and permutes;   */
/* the key is bumped by two Weyl increments (golden ratio, sqrt(3)-1) between  */
/* rounds.                                                                     */
/* ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t a = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t b = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t a_hi = (uint32_t)(a >> 32), a_lo = (uint32_t)a;
        uint32_t b_hi = (uint32_t)(b >> 32), b_lo = (uint32_t)b;
        uint32_t n0 = b_hi ^ c1 ^ k0;
        uint32_t n1 = b_lo;
        uint32_t n2 = a_hi ^ c3 ^ k1;
        uint32_t n3 = a_lo;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void draw_words(uint64_t seed, int64_t t, int32_t g, uint32_t w[4])
{
    uint32_t ctr[4] = { (uint32_t)g, 0u, (uint32_t)((uint64_t)t & 0xFFFFFFFFu),
                        (uint32_t)((uint64_t)t >> 32) };
    uint32_t key[2] = { (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32) };
    orc_philox4x32_10(ctr, key, w);
}

/* ------------------------------------------------------------------------- */
/* QAOA MaxCut circuit (Sec. "Quantum Approximate Optimization Algorithm")     */
/* ------------------------------------------------------------------------- */
int32_t orc_qaoa_gate_count(int32_t n, int32_t num_edges, int32_t p)
{
    return n + p * (num_edges + n);
}

int32_t orc_qaoa_gates(int32_t n, int32_t num_edges, const int32_t *edges, int32_t p,
                       const double *gammas, const double *betas, orc_gate *out)
{
    int32_t g = 0;
    for (int32_t q = 0; q < n; ++q) {
        out[g].kind = ORC_H; out[g].q0 = q; out[g].q1 = -1; out[g].angle = 0.0; ++g;
    }
    for (int32_t l = 0; l < p; ++l) {
        for (int32_t e = 0; e < num_edges; ++e) {
            out[g].kind = ORC_ZZ; out[g].q0 = edges[2 * e]; out[g].q1 = edges[2 * e + 1];
            out[g].angle = gammas[l]; ++g;
        }
        for (int32_t q = 0; q < n; ++q) {
            out[g].kind = ORC_RX; out[g].q0 = q; out[g].q1 = -1; out[g].angle = betas[l]; ++g;
        }
    }
    return g;
}

/* cut value C(x) = number of edges whose endpoints take different values. */
static double cut_value(uint64_t x, int32_t num_edges, const int32_t *edges)
{
    int c = 0;
    for (int32_t e = 0; e < num_edges; ++e)
        c += (int)(((x >> edges[2 * e]) ^ (x >> edges[2 * e + 1])) & 1u);
    return (double)c;
}

/* ------------------------------------------------------------------------- */
/* Noise probabilities and integer thresholds                                 */
/* ------------------------------------------------------------------------- */
/* Pauli probability of a 1q channel for gate type (1q) or of each qubit of a  */
/* product-mode 2q channel.                                                    */
static double pauli_total_1q(const orc_noise *nz, double x)
{
    return nz->param == 1 ? 0.75 * x : x;
}

/* probs[k] for Pauli code k: 4 entries for 1q gates, 16 for 2q gates. */
int32_t orc_pauli_probs(const orc_noise *nz, int32_t two_qubit, double *probs)
{
    if (!two_qubit) {
        double p = pauli_total_1q(nz, nz->p1);
        probs[0] = 1.0 - p;
        probs[1] = probs[2] = probs[3] = p / 3.0;
        return 4;
    }
    if (nz->twoq_mode == 1) {
        double p = pauli_total_1q(nz, nz->p2);
        double s[4] = { 1.0 - p, p / 3.0, p / 3.0, p / 3.0 };
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) probs[4 * a + b] = s[a] * s[b];
        return 16;
    }
    double p = nz->param == 1 ? (15.0 / 16.0) * nz->p2 : nz->p2;
    probs[0] = 1.0 - p;
    for (int k = 1; k < 16; ++k) probs[k] = p / 15.0;
    return 16;
}

/* T_k = floor(2^32 * c_k), c_k = probs[0] + ... + probs[k] summed in order. */
void orc_thresholds(const double *probs, int32_t count, uint64_t *thr)
{
    double c = 0.0;
    for (int32_t k = 0; k < count; ++k) {
        c += probs[k];
        double v = floor(c * 4294967296.0);
        if (v < 0.0) v = 0.0;
        if (v > 4294967296.0) v = 4294967296.0;
        thr[k] = (uint64_t)v;
    }
}

static int pick_code(uint32_t w, const uint64_t *thr, int32_t count)
{
    for (int32_t k = 0; k < count - 1; ++k)
        if ((uint64_t)w < thr[k]) return k;
    return count - 1;
}

/* ------------------------------------------------------------------------- */
/* State-vector primitives (complex128)                                       */
/* ------------------------------------------------------------------------- */
static void sv_apply_1q(cplx *psi, int32_t n, int32_t q, const cplx m[4])
{
    uint64_t dim = (uint64_t)1 << n, bit = (uint64_t)1 << q;
    for (uint64_t x = 0; x < dim; ++x) {
        if (x & bit) continue;
        cplx a = psi[x], b = psi[x | bit];
        psi[x] = m[0] * a + m[1] * b;
        psi[x | bit] = m[2] * a + m[3] * b;
    }
}

static void sv_apply_zz(cplx *psi, int32_t n, int32_t i, int32_t j, double gamma)
{
    uint64_t dim = (uint64_t)1 << n;
    cplx ph = cexp(-I * gamma);
    for (uint64_t x = 0; x < dim; ++x)
        if (((x >> i) ^ (x >> j)) & 1u) psi[x] *= ph;
}

static void pauli_matrix(int code, cplx m[4])
{
    switch (code) {
    case 0: m[0] = 1; m[1] = 0; m[2] = 0; m[3] = 1; break;   /* I */
    case 1: m[0] = 0; m[1] = 1; m[2] = 1; m[3] = 0; break;   /* X */
    case 2: m[0] = 0; m[1] = -I; m[2] = I; m[3] = 0; break;  /* Y */
    default: m[0] = 1; m[1] = 0; m[2] = 0; m[3] = -1; break; /* Z */
    }
}

static void gate_matrix_1q(const orc_gate *gt, cplx m[4])
{
    if (gt->kind == ORC_H) {
        double s = 1.0 / sqrt(2.0);
        m[0] = s; m[1] = s; m[2] = s; m[3] = -s;
    } else { /* exp(-i beta X) */
        double c = cos(gt->angle), s = sin(gt->angle);
        m[0] = c; m[1] = -I * s; m[2] = -I * s; m[3] = c;
    }
}

static void sv_apply_gate(cplx *psi, int32_t n, const orc_gate *gt)
{
    if (gt->kind == ORC_ZZ) {
        sv_apply_zz(psi, n, gt->q0, gt->q1, gt->angle);
    } else {
        cplx m[4];
        gate_matrix_1q(gt, m);
        sv_apply_1q(psi, n, gt->q0, m);
    }
}

static double sv_norm2(const cplx *psi, int32_t n)
{
    uint64_t dim = (uint64_t)1 << n;
    double s = 0.0;
    for (uint64_t x = 0; x < dim; ++x) s += creal(psi[x]) * creal(psi[x]) + cimag(psi[x]) * cimag(psi[x]);
    return s;
}

static double sv_weight_one(const cplx *psi, int32_t n, int32_t q)
{
    uint64_t dim = (uint64_t)1 << n, bit = (uint64_t)1 << q;
    double s = 0.0;
    for (uint64_t x = 0; x < dim; ++x)
        if (x & bit) s += creal(psi[x]) * creal(psi[x]) + cimag(psi[x]) * cimag(psi[x]);
    return s;
}

static void sv_scale(cplx *psi, int32_t n, double f)
{
    uint64_t dim = (uint64_t)1 << n;
    for (uint64_t x = 0; x < dim; ++x) psi[x] *= f;
}

/* Amplitude damping Kraus pair: K0 = [[1,0],[0,sqrt(1-g)]], K1 = [[0,sqrt(g)],[0,0]]. */
static void damping_kraus(double gamma, int which, cplx m[4])
{
    if (which == 0) { m[0] = 1; m[1] = 0; m[2] = 0; m[3] = sqrt(1.0 - gamma); }
    else            { m[0] = 0; m[1] = sqrt(gamma); m[2] = 0; m[3] = 0; }
}

/*
 * One trajectory.  If forced != NULL the branch bytes are taken from it instead
 * of being sampled, and *weight receives the product of the probabilities of the
 * chosen branches (the Born weight of this Kraus string).  branch byte of gate g:
 * Pauli code in bits 0..3, K1 on the first qubit in bit 4, K1 on the second in
 * bit 5.  Returns 0, or 1 if a forced branch has probability zero.
 */
static int traj_one(int32_t n, const orc_gate *gates, int32_t G, const orc_noise *nz,
                    uint64_t seed, int64_t t, const uint8_t *forced, cplx *psi,
                    uint8_t *branch_out, double *weight)
{
    uint64_t dim = (uint64_t)1 << n;
    double pr1[4], pr2[16];
    uint64_t th1[4], th2[16];
    orc_pauli_probs(nz, 0, pr1); orc_thresholds(pr1, 4, th1);
    orc_pauli_probs(nz, 1, pr2); orc_thresholds(pr2, 16, th2);
    memset(psi, 0, dim * sizeof(cplx));
    psi[0] = 1.0;
    double w_total = 1.0;
    for (int32_t g = 0; g < G; ++g) {
        const orc_gate *gt = &gates[g];
        int twoq = gt->kind == ORC_ZZ;
        sv_apply_gate(psi, n, gt);
        uint32_t w[4];
        draw_words(seed, t, g, w);
        int code = forced ? (forced[g] & 15) : pick_code(w[0], twoq ? th2 : th1, twoq ? 16 : 4);
        if (forced) w_total *= twoq ? pr2[code] : pr1[code];
        cplx m[4];
        if (twoq) {
            pauli_matrix(code >> 2, m); sv_apply_1q(psi, n, gt->q0, m);
            pauli_matrix(code & 3, m);  sv_apply_1q(psi, n, gt->q1, m);
        } else {
            pauli_matrix(code, m); sv_apply_1q(psi, n, gt->q0, m);
        }
        uint8_t rec = (uint8_t)code;
        if (nz->damping > 0.0) {
            int nq = twoq ? 2 : 1;
            for (int k = 0; k < nq; ++k) {
                int32_t q = k == 0 ? gt->q0 : gt->q1;
                double total = sv_norm2(psi, n);
                double p1 = nz->damping * sv_weight_one(psi, n, q) / total;
                int jump;
                if (forced) {
                    jump = (forced[g] >> (4 + k)) & 1;
                    w_total *= jump ? p1 : 1.0 - p1;
                    if ((jump ? p1 : 1.0 - p1) <= 0.0) return 1;
                } else {
                    double u = ((double)w[1 + k] + 0.5) * (1.0 / 4294967296.0);
                    jump = u < p1;
                }
                damping_kraus(nz->damping, jump, m);
                sv_apply_1q(psi, n, q, m);
                sv_scale(psi, n, 1.0 / sqrt(sv_norm2(psi, n)));
                if (jump) rec |= (uint8_t)(1u << (4 + k));
            }
        }
        if (branch_out) branch_out[g] = rec;
    }
    if (weight) *weight = w_total;
    return 0;
}

/*
 * Ensemble of trajectories t0 .. t0+count-1.
 *   amps      count x 2^n complex128, or NULL
 *   branches  count x G bytes, or NULL
 *   c_traj    count doubles: <C>_t = sum_x |psi_t,x|^2 C(x), or NULL
 *   probs_sum 2^n doubles, receives sum_t |psi_t|^2 (not divided by count), or NULL
 *   sums      2 doubles: sum_t <C>_t and sum_t <C>_t^2, or NULL
 */
int32_t orc_traj_run(int32_t n, int32_t num_edges, const int32_t *edges, const orc_gate *gates,
                     int32_t G, const orc_noise *nz, uint64_t seed, int64_t t0, int64_t count,
                     cplx *amps, uint8_t *branches, double *c_traj, double *probs_sum,
                     double *sums, int32_t threads)
{
    uint64_t dim = (uint64_t)1 << n;
    double *ct = (double *)malloc(sizeof(double) * (size_t)(count > 0 ? count : 1));
    if (!ct) return 2;
    int nthr = 1;
#ifdef _OPENMP
    nthr = threads > 0 ? threads : omp_get_max_threads();
#else
    (void)threads;
#endif
    double *pp = NULL;
    if (probs_sum) {
        pp = (double *)calloc((size_t)nthr * dim, sizeof(double));
        if (!pp) { free(ct); return 2; }
    }
    cplx *work = (cplx *)malloc((size_t)nthr * dim * sizeof(cplx));
    if (!work) { free(pp); free(ct); return 2; }
    int err = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthr)
#endif
    for (int64_t i = 0; i < count; ++i) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        cplx *psi = work + (size_t)tid * dim;
        traj_one(n, gates, G, nz, seed, t0 + i, NULL, psi,
                 branches ? branches + (size_t)i * (size_t)G : NULL, NULL);
        double c = 0.0;
        for (uint64_t x = 0; x < dim; ++x) {
            double pr = creal(psi[x]) * creal(psi[x]) + cimag(psi[x]) * cimag(psi[x]);
            c += pr * cut_value(x, num_edges, edges);
            if (pp) pp[(size_t)tid * dim + x] += pr;
        }
        ct[i] = c;
        if (amps) memcpy(amps + (size_t)i * dim, psi, dim * sizeof(cplx));
    }
    free(work);
    if (!err) {
        if (c_traj) memcpy(c_traj, ct, sizeof(double) * (size_t)count);
        if (sums) {
            double s1 = 0.0, s2 = 0.0;
            for (int64_t i = 0; i < count; ++i) { s1 += ct[i]; s2 += ct[i] * ct[i]; }
            sums[0] = s1; sums[1] = s2;
        }
        if (probs_sum) {
            for (uint64_t x = 0; x < dim; ++x) {
                double s = 0.0;
                for (int k = 0; k < nthr; ++k) s += pp[(size_t)k * dim + x];
                probs_sum[x] = s;
            }
        }
    }
    free(pp);
    free(ct);
    return err;
}

/* One trajectory with a forced Kraus string; see traj_one.  psi: 2^n complex128. */
int32_t orc_traj_forced(int32_t n, const orc_gate *gates, int32_t G, const orc_noise *nz,
                        const uint8_t *forced, cplx *psi, double *weight)
{
    return traj_one(n, gates, G, nz, 0, 0, forced, psi, NULL, weight);
}

/* ------------------------------------------------------------------------- */
/* Density-matrix primitives.  rho is 2^n x 2^n complex128, row-major.        */
/* ------------------------------------------------------------------------- */
/* rho <- M rho M^dagger for a 2x2 matrix M on qubit q (M need not be unitary). */
void orc_dm_apply_1q(cplx *rho, int32_t n, int32_t q, const cplx m[4])
{
    uint64_t dim = (uint64_t)1 << n, bit = (uint64_t)1 << q;
    cplx mc[4] = { conj(m[0]), conj(m[1]), conj(m[2]), conj(m[3]) };
#ifdef _OPENMP
#pragma omp parallel for schedule(static) if (n >= 8)
#endif
    for (int64_t r = 0; r < (int64_t)dim; ++r) { /* rows: rho <- rho M^dagger */
        cplx *row = rho + (uint64_t)r * dim;
        for (uint64_t c = 0; c < dim; ++c) {
            if (c & bit) continue;
            cplx a = row[c], b = row[c | bit];
            row[c] = a * mc[0] + b * mc[1];
            row[c | bit] = a * mc[2] + b * mc[3];
        }
    }
#ifdef _OPENMP
#pragma omp parallel for schedule(static) if (n >= 8)
#endif
    for (int64_t r = 0; r < (int64_t)dim; ++r) { /* columns: rho <- M rho */
        if ((uint64_t)r & bit) continue;
        cplx *r0 = rho + (uint64_t)r * dim, *r1 = rho + ((uint64_t)r | bit) * dim;
        for (uint64_t c = 0; c < dim; ++c) {
            cplx a = r0[c], b = r1[c];
            r0[c] = m[0] * a + m[1] * b;
            r1[c] = m[2] * a + m[3] * b;
        }
    }
}

static void dm_axpy(cplx *acc, const cplx *x, double w, uint64_t len)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(static) if (len >= 65536)
#endif
    for (int64_t k = 0; k < (int64_t)len; ++k) acc[k] += w * x[k];
}

/* E(rho) = sum_j K_j rho K_j^dagger with Pauli Kraus ops K_j = sqrt(w_j) P_j. */
static int dm_pauli_channel(cplx *rho, int32_t n, int32_t q0, int32_t q1, const double *w, int count)
{
    uint64_t dim = (uint64_t)1 << n, len = dim * dim;
    cplx *acc = (cplx *)calloc(len, sizeof(cplx));
    cplx *tmp = (cplx *)malloc(len * sizeof(cplx));
    if (!acc || !tmp) { free(acc); free(tmp); return 2; }
    for (int k = 0; k < count; ++k) {
        if (w[k] == 0.0) continue;
        memcpy(tmp, rho, len * sizeof(cplx));
        cplx m[4];
        if (count == 4) {
            pauli_matrix(k, m); orc_dm_apply_1q(tmp, n, q0, m);
        } else {
            pauli_matrix(k >> 2, m); orc_dm_apply_1q(tmp, n, q0, m);
            pauli_matrix(k & 3, m);  orc_dm_apply_1q(tmp, n, q1, m);
        }
        dm_axpy(acc, tmp, w[k], len);
    }
    memcpy(rho, acc, len * sizeof(cplx));
    free(acc); free(tmp);
    return 0;
}

/* 1q depolarizing channel with the Pauli probabilities of a 1q gate. */
int32_t orc_dm_depolarize_1q(cplx *rho, int32_t n, int32_t q, const orc_noise *nz)
{
    double w[4];
    orc_pauli_probs(nz, 0, w);
    return dm_pauli_channel(rho, n, q, -1, w, 4);
}

/* 2q channel of a ZZ gate (15-Pauli depolarizing or product mode). */
int32_t orc_dm_depolarize_2q(cplx *rho, int32_t n, int32_t q0, int32_t q1, const orc_noise *nz)
{
    double w[16];
    orc_pauli_probs(nz, 1, w);
    return dm_pauli_channel(rho, n, q0, q1, w, 16);
}

/* Amplitude damping on qubit q: K0 rho K0^dagger + K1 rho K1^dagger. */
int32_t orc_dm_damp(cplx *rho, int32_t n, int32_t q, double gamma)
{
    uint64_t dim = (uint64_t)1 << n, len = dim * dim;
    cplx *tmp = (cplx *)malloc(len * sizeof(cplx));
    if (!tmp) return 2;
    cplx k0[4], k1[4];
    damping_kraus(gamma, 0, k0);
    damping_kraus(gamma, 1, k1);
    memcpy(tmp, rho, len * sizeof(cplx));
    orc_dm_apply_1q(rho, n, q, k0);
    orc_dm_apply_1q(tmp, n, q, k1);
    dm_axpy(rho, tmp, 1.0, len);
    free(tmp);
    return 0;
}

/* rho <- U rho U^dagger for one circuit gate. */
void orc_dm_gate(cplx *rho, int32_t n, const orc_gate *gt)
{
    uint64_t dim = (uint64_t)1 << n;
    if (gt->kind == ORC_ZZ) {
        cplx ph = cexp(-I * gt->angle);
#ifdef _OPENMP
#pragma omp parallel for schedule(static) if (n >= 8)
#endif
        for (int64_t r = 0; r < (int64_t)dim; ++r) {
            cplx dr = (((uint64_t)r >> gt->q0) ^ ((uint64_t)r >> gt->q1)) & 1u ? ph : 1.0;
            for (uint64_t c = 0; c < dim; ++c) {
                cplx dc = ((c >> gt->q0) ^ (c >> gt->q1)) & 1u ? ph : 1.0;
                rho[(uint64_t)r * dim + c] *= dr * conj(dc);
            }
        }
    } else {
        cplx m[4];
        gate_matrix_1q(gt, m);
        orc_dm_apply_1q(rho, n, gt->q0, m);
    }
}

/*
 * Full noisy circuit on the density matrix.
 *   rho_out  2^n x 2^n complex128 (NULL: use internal storage)
 *   diag_out 2^n doubles = sigma_exact, or NULL
 *   c_out    Tr(rho C), or NULL
 */
int32_t orc_dm_run(int32_t n, int32_t num_edges, const int32_t *edges, const orc_gate *gates,
                   int32_t G, const orc_noise *nz, cplx *rho_out, double *diag_out, double *c_out)
{
    uint64_t dim = (uint64_t)1 << n, len = dim * dim;
    cplx *rho = rho_out ? rho_out : (cplx *)malloc(len * sizeof(cplx));
    if (!rho) return 2;
    memset(rho, 0, len * sizeof(cplx));
    rho[0] = 1.0;
    int err = 0;
    for (int32_t g = 0; g < G && !err; ++g) {
        const orc_gate *gt = &gates[g];
        orc_dm_gate(rho, n, gt);
        if (gt->kind == ORC_ZZ) err = orc_dm_depolarize_2q(rho, n, gt->q0, gt->q1, nz);
        else err = orc_dm_depolarize_1q(rho, n, gt->q0, nz);
        if (!err && nz->damping > 0.0) {
            err = orc_dm_damp(rho, n, gt->q0, nz->damping);
            if (!err && gt->kind == ORC_ZZ) err = orc_dm_damp(rho, n, gt->q1, nz->damping);
        }
    }
    if (!err) {
        double c = 0.0;
        for (uint64_t x = 0; x < dim; ++x) {
            double d = creal(rho[x * dim + x]);
            if (diag_out) diag_out[x] = d;
            c += d * cut_value(x, num_edges, edges);
        }
        if (c_out) *c_out = c;
    }
    if (!rho_out) free(rho);
    return err;
}

/* Error = 1 - (sum_x sqrt(sa_x se_x))^2  (Sec. "Stochastic Noise Implementation", Eq. 1). */
double orc_error(const double *sa, const double *se, int64_t len)
{
    double s = 0.0;
    for (int64_t x = 0; x < len; ++x) s += sqrt(sa[x] * se[x]);
    return 1.0 - s * s;
}
