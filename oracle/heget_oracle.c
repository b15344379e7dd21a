/*
 * heget_oracle.c -- plain, slow, FP64 CPU oracle for u ubar -> n photons.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only the tests, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py use it.  It shares no code, header, table or
 * constant generator with the CUDA library.
 *
 * What it computes is the plain definition of the paper's method
 * (Hagiwara et al., "Fast calculation of HELAS amplitudes using graphics
 * processing unit (GPU)", arXiv:0908.4403):
 *
 *   - Sec. 2.1, eqs. (6)-(8): the helicity amplitude of
 *     q(p1,s1) qbar(p2,s2) -> gamma(k1,l1) ... gamma(kn,ln) as the sum over all
 *     n! photon orderings of one fermion-line chain
 *         vbar(p2) [eps*_{pn} S(q_{n-1}) ... S(q_1) eps*_{p1}] u(p1) (eQ)^n,
 *     S(q) = qslash / q^2,  q_l = p1 - sum_{m<=l} k_{pi(m)},
 *     evaluated with explicit 4x4 Dirac matrices in the chiral basis, every
 *     ordering computed from scratch (no prefix sharing);
 *   - Sec. 2.1, eq. (2): the sum over all 2^(n+2) helicity combinations and the
 *     colour / spin / identical-particle factors of the partonic cross section;
 *   - Sec. 2.1, eq. (4): flat massless n-body phase space, generated with RAMBO
 *     (Kleiss, Stirling, Ellis, Comput. Phys. Commun. 40 (1986) 359), the
 *     generator the paper leaves unnamed (Sec. 3 only says that the kernel
 *     turns random numbers into a phase-space point and its weight);
 *   - Sec. 2.2, eqs. (9)-(10): the photon cuts.
 *
 * External states follow the textbook helicity construction in the chiral
 * basis; they agree with the HELAS-convention wave functions of Sec. 4 and
 * Appendix B (ixxxx*, oxxxx*, vxxxx*) up to phases, which drop out of |M|^2:
 *   u(p,+) = sqrt(2E) (0, 0, xi+),   u(p,-) = sqrt(2E) (xi-, 0, 0),
 *   xi+ = (cos th/2, e^{i ph} sin th/2),  xi- = (-e^{-i ph} sin th/2, cos th/2),
 *   v(p,l) = u(p,-l),   vbar = v^dagger gamma^0,
 *   eps(k,l) = (0; -l e_theta - i e_phi)/sqrt2   (used conjugated: outgoing),
 * i.e. the light-cone gauge eps.n = 0 with n = (k0, -kvec) of Sec. 4.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11),
 * implemented here from its published definition.
 *
 * Every floating-point quantity is IEEE double; build with -ffp-contract=off.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cx;

#define ORACLE_MAXN 8
#define ORACLE_MAXP (ORACLE_MAXN + 2)

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator (Salmon et al., SC'11, Sec. 2-3)   */
/* ------------------------------------------------------------------------ */

void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                          uint32_t out[4])
{
    /* round multipliers and Weyl key increments from the Philox paper */
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t a = (uint64_t)M0 * (uint64_t)x0;
        uint64_t b = (uint64_t)M1 * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(b >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)b;
        uint32_t y2 = (uint32_t)(a >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)a;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/*
 * Uniform number number `draw` of stream `stream` for phase-space point
 * `point` under `seed`.  Counter = (point lo, point hi, draw/2, stream),
 * key = (seed lo, seed hi).  Draw d uses output words (2(d&1), 2(d&1)+1):
 * m = ((w_hi << 32) | w_lo) >> 12 (52 bits), u = (m + 1/2) 2^-52, exact in
 * FP64 and strictly inside (0,1).
 */
double oracle_uniform(uint64_t seed, uint64_t point, uint32_t stream,
                      uint32_t draw)
{
    uint32_t ctr[4] = {(uint32_t)point, (uint32_t)(point >> 32), draw >> 1,
                       stream};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    oracle_philox4x32_10(ctr, key, w);
    uint32_t lo = w[2 * (draw & 1u)], hi = w[2 * (draw & 1u) + 1];
    uint64_t m = ((((uint64_t)hi) << 32) | (uint64_t)lo) >> 12;
    return ((double)m + 0.5) * 0x1p-52;
}

#define STREAM_SQRTS 0u
#define STREAM_RAMBO 1u

/* ------------------------------------------------------------------------ */
/* Dirac algebra: chiral basis, gamma5 = diag(-1,-1,+1,+1)                  */
/* (the block convention of Sec. 4 / Appendix B.3: P_L acts on comps 0,1)   */
/* ------------------------------------------------------------------------ */

typedef struct { cx m[4][4]; } mat4;
typedef struct { cx v[4]; } spin4;

static mat4 G[4];           /* gamma^mu, mu = 0..3 (upper index) */
static int g_ready = 0;

static void init_gammas(void)
{
    if (g_ready) return;
    memset(G, 0, sizeof G);
    /* sigma^i */
    cx s[4][2][2];
    memset(s, 0, sizeof s);
    s[0][0][0] = 1; s[0][1][1] = 1;                 /* identity */
    s[1][0][1] = 1; s[1][1][0] = 1;                 /* sigma_x */
    s[2][0][1] = -I; s[2][1][0] = I;                /* sigma_y */
    s[3][0][0] = 1; s[3][1][1] = -1;                /* sigma_z */
    /* gamma^0 = [[0,1],[1,0]],  gamma^i = [[0, sigma^i], [-sigma^i, 0]] */
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            G[0].m[a][2 + b] = s[0][a][b];
            G[0].m[2 + a][b] = s[0][a][b];
            for (int i = 1; i <= 3; ++i) {
                G[i].m[a][2 + b] = s[i][a][b];
                G[i].m[2 + a][b] = -s[i][a][b];
            }
        }
    g_ready = 1;
}

/* aslash = gamma^mu a_mu = gamma^0 a^0 - gamma^i a^i  (metric +,-,-,-) */
static mat4 slash(const cx a[4])
{
    mat4 r;
    for (int x = 0; x < 4; ++x)
        for (int y = 0; y < 4; ++y)
            r.m[x][y] = G[0].m[x][y] * a[0] - G[1].m[x][y] * a[1]
                      - G[2].m[x][y] * a[2] - G[3].m[x][y] * a[3];
    return r;
}

static spin4 matvec(const mat4* A, const spin4* v)
{
    spin4 r;
    for (int x = 0; x < 4; ++x) {
        cx acc = 0;
        for (int y = 0; y < 4; ++y) acc += A->m[x][y] * v->v[y];
        r.v[x] = acc;
    }
    return r;
}

static mat4 mat_scale(const mat4* A, double c)
{
    mat4 r;
    for (int x = 0; x < 4; ++x)
        for (int y = 0; y < 4; ++y) r.m[x][y] = A->m[x][y] * c;
    return r;
}

static double mdot(const double a[4], const double b[4])
{
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
}

/* ------------------------------------------------------------------------ */
/* External states (textbook helicity states; phases differ from HELAS)     */
/* ------------------------------------------------------------------------ */

/* polar angles of a 3-momentum; phi := 0 when pT = 0 (atan2(0,0) = 0) */
static void angles(const double p[4], double* cth, double* sth_half,
                   double* cth_half, double* phi)
{
    double pabs = sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
    double c = p[3] / pabs;
    if (c > 1) c = 1;
    if (c < -1) c = -1;
    *cth = c;
    *cth_half = sqrt((1 + c) / 2);
    *sth_half = sqrt((1 - c) / 2);
    *phi = atan2(p[2], p[1]);
}

/* u(p, lam) for a massless fermion, lam = +1 / -1 */
static spin4 u_spinor(const double p[4], int lam)
{
    double c, sh, ch, ph;
    angles(p, &c, &sh, &ch, &ph);
    double nrm = sqrt(2 * p[0]);
    spin4 u = {{0, 0, 0, 0}};
    if (lam > 0) {          /* right-handed: lower block = xi+ */
        u.v[2] = nrm * ch;
        u.v[3] = nrm * cexp(I * ph) * sh;
    } else {                /* left-handed: upper block = xi- */
        u.v[0] = -nrm * cexp(-I * ph) * sh;
        u.v[1] = nrm * ch;
    }
    return u;
}

/* vbar(p, lam) = v^dagger gamma^0 with v(p, lam) = u(p, -lam); as a row */
static spin4 vbar_spinor(const double p[4], int lam)
{
    spin4 v = u_spinor(p, -lam);
    spin4 r;
    /* (v^dagger gamma^0)_y = sum_x conj(v_x) gamma^0_{x y} */
    for (int y = 0; y < 4; ++y) {
        cx acc = 0;
        for (int x = 0; x < 4; ++x) acc += conj(v.v[x]) * G[0].m[x][y];
        r.v[y] = acc;
    }
    return r;
}

/* eps(k, lam) = (0; -lam e_theta - i e_phi)/sqrt2 */
static void eps_vector(const double k[4], int lam, cx e[4])
{
    double c, sh, ch, ph;
    angles(k, &c, &sh, &ch, &ph);
    double s = sqrt(1 - c * c);
    double cp = cos(ph), sp = sin(ph);
    double eth[3] = {c * cp, c * sp, -s};
    double ephi[3] = {-sp, cp, 0};
    e[0] = 0;
    for (int i = 0; i < 3; ++i)
        e[i + 1] = (-lam * eth[i] - I * ephi[i]) / sqrt(2.0);
}

/* ------------------------------------------------------------------------ */
/* Amplitude of Sec. 2.1, eqs. (6)-(8)                                       */
/* ------------------------------------------------------------------------ */

typedef struct {
    double alpha;   /* fine-structure constant */
    double Q;       /* quark charge in units of e */
} oracle_couplings;

static int next_permutation(int* a, int n)
{
    int i = n - 2;
    while (i >= 0 && a[i] >= a[i + 1]) --i;
    if (i < 0) return 0;
    int j = n - 1;
    while (a[j] <= a[i]) --j;
    int t = a[i]; a[i] = a[j]; a[j] = t;
    for (int l = i + 1, r = n - 1; l < r; ++l, --r) {
        t = a[l]; a[l] = a[r]; a[r] = t;
    }
    return 1;
}

/* Neumaier compensated sum of complex terms */
typedef struct { double s_re, c_re, s_im, c_im; } csum;

static void csum_add(csum* S, cx x)
{
    double v[2] = {creal(x), cimag(x)};
    double* s[2] = {&S->s_re, &S->s_im};
    double* c[2] = {&S->c_re, &S->c_im};
    for (int k = 0; k < 2; ++k) {
        double t = *s[k] + v[k];
        if (fabs(*s[k]) >= fabs(v[k])) *c[k] += (*s[k] - t) + v[k];
        else *c[k] += (v[k] - t) + *s[k];
        *s[k] = t;
    }
}

static cx csum_value(const csum* S)
{
    return (S->s_re + S->c_re) + I * (S->s_im + S->c_im);
}

/*
 * One chain for photon ordering `perm` with photon vertices given as matrices
 * V[i] (= eps*_i slash, or gamma^mu, or k_i slash / k_i^0):
 *   vbar(p2) V[perm[n-1]] S(q_{n-1}) ... S(q_1) V[perm[0]] u(p1),
 * evaluated as matrix-vector products onto u(p1).
 */
static cx chain(int n, const double* mom, const int* perm, const mat4* V,
                const spin4* u1, const spin4* vb2)
{
    const double* p1 = mom;
    spin4 psi = *u1;
    double q[4] = {p1[0], p1[1], p1[2], p1[3]};
    for (int l = 0; l < n; ++l) {
        psi = matvec(&V[perm[l]], &psi);
        if (l == n - 1) break;
        const double* k = mom + 4 * (2 + perm[l]);
        for (int mu = 0; mu < 4; ++mu) q[mu] -= k[mu];
        cx qc[4] = {q[0], q[1], q[2], q[3]};
        mat4 S = slash(qc);
        S = mat_scale(&S, 1.0 / mdot(q, q));
        psi = matvec(&S, &psi);
    }
    cx a = 0;
    for (int x = 0; x < 4; ++x) a += vb2->v[x] * psi.v[x];
    return a;
}

/*
 * Helicity amplitude M_h (Sec. 2.1, eq. (6)): the sum over all n! orderings.
 * Helicity index h: bit0 = s1 (1 -> +), bit1 = s2, bit(2+i) = lambda_{i+1}.
 * mom: (n+2) x 4 doubles, order p1, p2, k1..kn, components (E, px, py, pz).
 * ward >= 0 replaces the polarisation of photon `ward` by k/k^0.
 * sum_abs (may be NULL) receives sum_pi |A_pi| (condition estimate).
 */
static cx amplitude(int n, const double* mom, int h, int ward,
                    const oracle_couplings* cpl, double* sum_abs)
{
    init_gammas();
    int s1 = (h & 1) ? 1 : -1, s2 = (h & 2) ? 1 : -1;
    spin4 u1 = u_spinor(mom, s1);
    spin4 vb2 = vbar_spinor(mom + 4, s2);
    mat4 V[ORACLE_MAXN];
    for (int i = 0; i < n; ++i) {
        const double* k = mom + 4 * (2 + i);
        cx e[4];
        if (i == ward) {
            for (int mu = 0; mu < 4; ++mu) e[mu] = k[mu] / k[0];
        } else {
            int lam = (h >> (2 + i)) & 1 ? 1 : -1;
            eps_vector(k, lam, e);
            for (int mu = 0; mu < 4; ++mu) e[mu] = conj(e[mu]);
        }
        V[i] = slash(e);
    }
    int perm[ORACLE_MAXN];
    for (int i = 0; i < n; ++i) perm[i] = i;
    csum S = {0, 0, 0, 0};
    double sabs = 0;
    do {
        cx a = chain(n, mom, perm, V, &u1, &vb2);
        csum_add(&S, a);
        sabs += cabs(a);
    } while (next_permutation(perm, n));
    double e = sqrt(4 * M_PI * cpl->alpha);
    double g = pow(e * cpl->Q, n);
    if (sum_abs) *sum_abs = sabs * g;
    return csum_value(&S) * g;
}

static int mask_bit(const uint32_t* mask, int h)
{
    if (!mask) return 1;
    return (mask[h >> 5] >> (h & 31)) & 1u;
}

/* sum over helicities in `mask` (NULL = all 2^(n+2)) of |M_h|^2 */
double oracle_amp2_point(int n, const double* mom, const uint32_t* mask,
                         double alpha, double Q)
{
    oracle_couplings cpl = {alpha, Q};
    double acc = 0;
    for (int h = 0; h < (1 << (n + 2)); ++h) {
        if (!mask_bit(mask, h)) continue;
        cx m = amplitude(n, mom, h, -1, &cpl, NULL);
        acc += creal(m) * creal(m) + cimag(m) * cimag(m);
    }
    return acc;
}

void oracle_amp2(int n, int64_t N, const double* mom, const uint32_t* mask,
                 double alpha, double Q, int threads, double* out)
{
    (void)threads;
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads > 0 ? threads : 1)
    for (int64_t i = 0; i < N; ++i)
        out[i] = oracle_amp2_point(n, mom + i * 4 * (n + 2), mask, alpha, Q);
}

/* complex helicity amplitude M_h (re, im) and sum_pi |A_pi| */
void oracle_amp_hel(int n, const double* mom, int h, int ward, double alpha,
                    double Q, double* re, double* im, double* sum_abs)
{
    oracle_couplings cpl = {alpha, Q};
    cx m = amplitude(n, mom, h, ward, &cpl, sum_abs);
    *re = creal(m);
    *im = cimag(m);
}

/*
 * Second route to sum_h |M_h|^2 with no polarisation vectors:
 * sum_lambda eps_mu eps*_nu -> -g_{mu nu} for each photon (valid for the full,
 * gauge-invariant sum over orderings), so
 *   sum_h |M_h|^2 = sum_{s1,s2} sum_{mu_1..mu_n} prod_i (-g_{mu_i mu_i})
 *                   |M^{mu_1..mu_n}_{s1 s2}|^2,
 * where M^{mu...} is the ordering sum with gamma^{mu_i} at photon i.
 */
double oracle_amp2_metric(int n, const double* mom, double alpha, double Q)
{
    init_gammas();
    double e = sqrt(4 * M_PI * alpha);
    double g = pow(e * Q, n);
    double total = 0;
    for (int sq = 0; sq < 4; ++sq) {
        int s1 = (sq & 1) ? 1 : -1, s2 = (sq & 2) ? 1 : -1;
        spin4 u1 = u_spinor(mom, s1);
        spin4 vb2 = vbar_spinor(mom + 4, s2);
        int nmu = 1 << (2 * n);
        for (int code = 0; code < nmu; ++code) {
            mat4 V[ORACLE_MAXN];
            double sign = 1;
            for (int i = 0; i < n; ++i) {
                int mu = (code >> (2 * i)) & 3;
                V[i] = G[mu];
                sign *= (mu == 0) ? -1.0 : 1.0;
            }
            int perm[ORACLE_MAXN];
            for (int i = 0; i < n; ++i) perm[i] = i;
            csum S = {0, 0, 0, 0};
            do {
                csum_add(&S, chain(n, mom, perm, V, &u1, &vb2));
            } while (next_permutation(perm, n));
            cx m = csum_value(&S) * g;
            total += sign * (creal(m) * creal(m) + cimag(m) * cimag(m));
        }
    }
    return total;
}

/* ------------------------------------------------------------------------ */
/* Phase space: RAMBO (Kleiss, Stirling, Ellis 1986), Sec. 2.1 eq. (4)      */
/* ------------------------------------------------------------------------ */

/* flat massless n-body phase-space volume in the normalisation of eq. (4) */
double oracle_phase_space_volume(int n, double s)
{
    double fact1 = 1, fact2 = 1;
    for (int i = 2; i <= n - 1; ++i) fact1 *= i;
    for (int i = 2; i <= n - 2; ++i) fact2 *= i;
    return pow(2 * M_PI, 4 - 3 * n) * pow(M_PI / 2, n - 1) * pow(s, n - 2)
           / (fact1 * fact2);
}

/*
 * RAMBO for n massless momenta at total energy sqrt_s in the CM frame.
 * r: 4n uniforms; photon i uses r[4i..4i+3] as
 *   cos(theta) = 2 r0 - 1,  phi = 2 pi r1,  q0 = -ln(r2 r3).
 * out: n x 4 doubles.  Returns the (constant) weight Phi_n(s).
 */
double oracle_rambo(int n, double sqrt_s, const double* r, double* out)
{
    double q[ORACLE_MAXN][4];
    double Q[4] = {0, 0, 0, 0};
    for (int i = 0; i < n; ++i) {
        double c = 2 * r[4 * i] - 1;
        double ph = 2 * M_PI * r[4 * i + 1];
        double q0 = -log(r[4 * i + 2] * r[4 * i + 3]);
        double s = sqrt(1 - c * c);
        q[i][0] = q0;
        q[i][1] = q0 * s * cos(ph);
        q[i][2] = q0 * s * sin(ph);
        q[i][3] = q0 * c;
        for (int mu = 0; mu < 4; ++mu) Q[mu] += q[i][mu];
    }
    double M = sqrt(mdot(Q, Q));
    double b[3] = {-Q[1] / M, -Q[2] / M, -Q[3] / M};
    double gam = Q[0] / M;
    double a = 1 / (1 + gam);
    double x = sqrt_s / M;
    for (int i = 0; i < n; ++i) {
        double bq = b[0] * q[i][1] + b[1] * q[i][2] + b[2] * q[i][3];
        out[4 * i] = x * (gam * q[i][0] + bq);
        for (int k = 0; k < 3; ++k)
            out[4 * i + 1 + k] = x * (q[i][1 + k] + b[k] * q[i][0] + a * bq * b[k]);
    }
    return oracle_phase_space_volume(n, sqrt_s * sqrt_s);
}

/* ------------------------------------------------------------------------ */
/* sqrt(s-hat) samplers, cuts, and per-point event generation               */
/* ------------------------------------------------------------------------ */

typedef struct {
    int kind;            /* 0 fixed, 1 uniform in [lo, hi], 2 toy PDF */
    double sqrt_s;       /* kind 0 */
    double lo, hi;       /* kind 1 */
    double e_beam;       /* kind 2: hadronic sqrt(s) = 2 e_beam */
    double a, b;         /* kind 2: density of x ~ x^a (1-x)^b, a = -1/2, b = 3 */
    double floor;        /* kind 2: accept if sqrt(s-hat) > floor */
    int max_tries;       /* rejection bound per loop */
} oracle_sampler;

typedef struct {
    double pt_min, eta_max, dr_min;   /* dr_min <= 0 disables the Delta R cut */
} oracle_cuts;

/*
 * Toy-PDF draw of one momentum fraction by rejection: proposal x = u^2 has
 * density ~ x^{-1/2}; accept with probability (1-x)^3.  Only a = -1/2 is
 * supported (checked by the caller).  Returns -1 if the bound is hit.
 */
static double draw_x(uint64_t seed, uint64_t i, uint32_t* d, double b, int max_tries)
{
    for (int t = 0; t < max_tries; ++t) {
        double u = oracle_uniform(seed, i, STREAM_SQRTS, (*d)++);
        double v = oracle_uniform(seed, i, STREAM_SQRTS, (*d)++);
        double x = u * u;
        if (v < pow(1 - x, b)) return x;
    }
    return -1;
}

/*
 * sqrt(s-hat) and boost rapidity y for point i.  Returns the number of outer
 * attempts used (toy PDF) or 1; *ok = 0 if a rejection bound was hit.
 */
static int sample_sqrt_s(const oracle_sampler* S, uint64_t seed, uint64_t i,
                         double* sqrt_s, double* y, int* ok)
{
    *ok = 1;
    *y = 0;
    if (S->kind == 0) { *sqrt_s = S->sqrt_s; return 1; }
    if (S->kind == 1) {
        double u = oracle_uniform(seed, i, STREAM_SQRTS, 0);
        *sqrt_s = S->lo + (S->hi - S->lo) * u;
        return 1;
    }
    uint32_t d = 0;
    for (int t = 1; t <= S->max_tries; ++t) {
        double x1 = draw_x(seed, i, &d, S->b, S->max_tries);
        double x2 = x1 < 0 ? -1 : draw_x(seed, i, &d, S->b, S->max_tries);
        if (x1 < 0 || x2 < 0) break;
        double rs = 2 * S->e_beam * sqrt(x1 * x2);
        if (rs > S->floor) {
            *sqrt_s = rs;
            *y = 0.5 * log(x1 / x2);
            return t;
        }
    }
    *ok = 0;
    *sqrt_s = S->kind == 2 ? S->floor : 0;
    return S->max_tries;
}

/* Sec. 2.2 eqs. (9)-(10); eta = asinh(pz/pT) + y (lab frame), strict cuts */
static int pass_cuts(int n, const double* k, double y, const oracle_cuts* C)
{
    double eta[ORACLE_MAXN], phi[ORACLE_MAXN];
    for (int i = 0; i < n; ++i) {
        const double* p = k + 4 * i;
        double pt = sqrt(p[1] * p[1] + p[2] * p[2]);
        if (!(pt > C->pt_min)) return 0;
        eta[i] = asinh(p[3] / pt) + y;
        if (!(fabs(eta[i]) < C->eta_max)) return 0;
        phi[i] = atan2(p[2], p[1]);
    }
    if (C->dr_min > 0) {
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) {
                double dphi = fabs(phi[i] - phi[j]);
                if (dphi > M_PI) dphi = 2 * M_PI - dphi;
                double deta = eta[i] - eta[j];
                if (!(sqrt(deta * deta + dphi * dphi) > C->dr_min)) return 0;
            }
    }
    return 1;
}

/* exported cut decision for one set of photon momenta (n x 4) */
int oracle_pass_cuts(int n, const double* k, double y, const oracle_cuts* C)
{
    return pass_cuts(n, k, y, C);
}

/*
 * Event generation for points i0 .. i0+N-1: sqrt(s-hat) sampling, RAMBO in
 * the partonic CM frame, incoming p1 = (rs/2)(1,0,0,1), p2 = (rs/2)(1,0,0,-1).
 * Any output pointer may be NULL.
 */
void oracle_phase_space(int n, uint64_t seed, int64_t i0, int64_t N,
                        const oracle_sampler* S, const oracle_cuts* C,
                        double* mom, double* weight, double* sqrt_s_out,
                        double* y_out, uint8_t* mask_out, int32_t* tries_out)
{
    for (int64_t j = 0; j < N; ++j) {
        uint64_t i = (uint64_t)(i0 + j);
        double rs, y;
        int ok;
        int tries = sample_sqrt_s(S, seed, i, &rs, &y, &ok);
        double r[4 * ORACLE_MAXN];
        for (int d = 0; d < 4 * n; ++d)
            r[d] = oracle_uniform(seed, i, STREAM_RAMBO, (uint32_t)d);
        double p[4 * ORACLE_MAXP];
        p[0] = rs / 2; p[1] = 0; p[2] = 0; p[3] = rs / 2;
        p[4] = rs / 2; p[5] = 0; p[6] = 0; p[7] = -rs / 2;
        double w = oracle_rambo(n, rs, r, p + 8);
        int pass = ok && (C ? pass_cuts(n, p + 8, y, C) : 1);
        if (mom) memcpy(mom + j * 4 * (n + 2), p, sizeof(double) * 4 * (n + 2));
        if (weight) weight[j] = ok ? w : 0;
        if (sqrt_s_out) sqrt_s_out[j] = rs;
        if (y_out) y_out[j] = y;
        if (mask_out) mask_out[j] = (uint8_t)pass;
        if (tries_out) tries_out[j] = tries;
    }
}

/* ------------------------------------------------------------------------ */
/* Cross-section weight, Sec. 2.1 eq. (2)                                   */
/* ------------------------------------------------------------------------ */

#define GEV2_TO_FB 0.3893793721e12   /* (hbar c)^2 = 0.3893793721 GeV^2 mb */

/*
 * dsigma-hat weight of one event in fb:
 *   (1/2s)(1/2^2)(1/3^2) 3 sum_h |M_h|^2 (1/n!) Phi_n(s) * mask.
 */
double oracle_event_weight(int n, double s, double amp2, double phi_n, int mask)
{
    double nfact = 1;
    for (int i = 2; i <= n; ++i) nfact *= i;
    if (!mask) return 0;
    return (1.0 / (2 * s)) * (1.0 / 4) * (1.0 / 9) * 3 * amp2 / nfact * phi_n
           * GEV2_TO_FB;
}

/*
 * Per-event weights w_i for points i0 .. i0+N-1 (the |M|^2 of points failing
 * the cuts is not needed and is skipped here; their weight is 0).
 */
void oracle_event_weights(int n, uint64_t seed, int64_t i0, int64_t N,
                          const oracle_sampler* S, const oracle_cuts* C,
                          double alpha, double Q, int threads, double* w_out,
                          uint8_t* mask_out, int32_t* tries_out)
{
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads > 0 ? threads : 1)
    for (int64_t j = 0; j < N; ++j) {
        double p[4 * ORACLE_MAXP], wps, rs, y;
        uint8_t m;
        int32_t t;
        oracle_phase_space(n, seed, i0 + j, 1, S, C, p, &wps, &rs, &y, &m, &t);
        double a2 = m ? oracle_amp2_point(n, p, NULL, alpha, Q) : 0;
        w_out[j] = oracle_event_weight(n, rs * rs, a2, wps, m);
        if (mask_out) mask_out[j] = m;
        if (tries_out) tries_out[j] = t;
    }
}

/*
 * Weighted histograms of kinematic observables of the generated events
 * (Sec. 5, Fig. 2: the largest photon transverse momentum and the photons'
 * Delta R separations).  Observables, with pT = sqrt(px^2 + py^2),
 * eta = asinh(pz / pT) + y (lab frame, as for the cuts of Sec. 2.2),
 * phi = atan2(py, px) and Delta phi folded into [0, pi]:
 *   0 the largest pT of the event's photons   (1 entry per event)
 *   1 the pT of each photon                   (n entries)
 *   2 the eta of each photon                  (n entries)
 *   3 Delta R of each photon pair             (n(n-1)/2 entries)
 *   4 the smallest Delta R of the event       (1 entry)
 *   5 sqrt(s-hat) = E1 + E2                   (1 entry)
 * Bins: 0 takes x < lo (and NaN), 1..nbins the uniform bins of [lo, hi)
 * (closed on the left), nbins + 1 takes x >= hi; x falls in bin
 * 1 + floor((x - lo) * (nbins / (hi - lo))).  Each entry adds the event's
 * weight w to the bin's sum of w and w^2 to its sum of w^2, both summed
 * with Neumaier's compensation.  out, per spec and bin in order:
 * (sum w, sum w^2).  mom: [N][n+2][4]; y: [N].
 */
typedef struct {
    int kind, nbins;
    double lo, hi;
} oracle_hist_spec;

typedef struct { double s, c; } nsum;   /* Neumaier sum */

static void nsum_add(nsum* a, double x)
{
    const double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}

static int hist_bin(double x, const oracle_hist_spec* H)
{
    if (!(x >= H->lo)) return 0;
    const double t = (x - H->lo) * ((double)H->nbins / (H->hi - H->lo));
    if (t >= H->nbins) return H->nbins + 1;
    return 1 + (int)t;
}

void oracle_hist(int n, int64_t N, const double* mom, const double* y, const double* w,
                 int nspec, const oracle_hist_spec* specs, double* out)
{
    int total = 0;
    for (int s = 0; s < nspec; ++s) total += specs[s].nbins + 2;
    nsum* sw = calloc((size_t)total, sizeof(nsum));
    nsum* sw2 = calloc((size_t)total, sizeof(nsum));
    for (int64_t j = 0; j < N; ++j) {
        const double* ev = mom + (size_t)j * (n + 2) * 4;
        const double* k = ev + 8;
        double pt[ORACLE_MAXN], eta[ORACLE_MAXN], phi[ORACLE_MAXN];
        for (int i = 0; i < n; ++i) {
            pt[i] = sqrt(k[4 * i + 1] * k[4 * i + 1] + k[4 * i + 2] * k[4 * i + 2]);
            eta[i] = asinh(k[4 * i + 3] / pt[i]) + y[j];
            phi[i] = atan2(k[4 * i + 2], k[4 * i + 1]);
        }
        double dr[ORACLE_MAXN * ORACLE_MAXN];
        int npair = 0;
        for (int a = 0; a < n; ++a)
            for (int b = a + 1; b < n; ++b) {
                double dphi = fabs(phi[a] - phi[b]);
                if (dphi > M_PI) dphi = 2 * M_PI - dphi;
                const double deta = eta[a] - eta[b];
                dr[npair++] = sqrt(deta * deta + dphi * dphi);
            }
        int off = 0;
        for (int s = 0; s < nspec; ++s) {
            const oracle_hist_spec* H = &specs[s];
            double x[ORACLE_MAXN * ORACLE_MAXN];
            int m = 0;
            switch (H->kind) {
                case 0:
                    x[0] = pt[0];
                    for (int i = 1; i < n; ++i)
                        if (pt[i] > x[0]) x[0] = pt[i];
                    m = 1;
                    break;
                case 1:
                    for (int i = 0; i < n; ++i) x[m++] = pt[i];
                    break;
                case 2:
                    for (int i = 0; i < n; ++i) x[m++] = eta[i];
                    break;
                case 3:
                    for (int p = 0; p < npair; ++p) x[m++] = dr[p];
                    break;
                case 4:
                    x[0] = dr[0];
                    for (int p = 1; p < npair; ++p)
                        if (dr[p] < x[0]) x[0] = dr[p];
                    m = npair > 0 ? 1 : 0;
                    break;
                default:
                    x[0] = ev[0] + ev[4];
                    m = 1;
                    break;
            }
            for (int e = 0; e < m; ++e) {
                const int b = off + hist_bin(x[e], H);
                nsum_add(&sw[b], w[j]);
                nsum_add(&sw2[b], w[j] * w[j]);
            }
            off += H->nbins + 2;
        }
    }
    for (int b = 0; b < total; ++b) {
        out[2 * b] = sw[b].s + sw[b].c;
        out[2 * b + 1] = sw2[b].s + sw2[b].c;
    }
    free(sw);
    free(sw2);
}
