/*
 * fmm_oracle.c -- plain, slow, FP64 CPU oracle for the M2L / FGT translation path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  It shares
 * no code, header, table or helper with the CUDA library in
 * paper_1009_3457_gb300/csrc, and neither side includes the other.
 *
 * Every routine is the paper's definition written out with plain loops, in
 * the paper's order, with no blocking, fusion or reordering:
 *
 *   Cruz, Layton & Barba, "How to obtain efficient GPU kernels: an
 *   illustration using FMM & FGT algorithms" (arXiv:1009.3457).
 *
 *   - FMM stages (initialisation, upward sweep, downward sweep, far field,
 *     near field): Sec. 2.1.
 *   - Downward-sweep steps (interaction list, M2L per list entry, reduction
 *     by summation): Sec. 4.1.
 *   - M2L matrix a_nk = (-1)^n C(n+k,k) (x_i - x_j)^(-k-n-1): Eq. (M2Lmat),
 *     Sec. 4.1, with x_i the target centre and x_j the source centre.
 *   - FGT Hermite / Taylor / Hermite-to-Taylor series: Eqs. (A_alpha),
 *     (B_beta), (C_beta), (hermite), (taylor), Sec. 2.2.
 *
 * Readings where the paper is silent or garbled (numbered as in the design
 * notes; R6, R10 and R11 concern the CUDA side, the error metric and the op
 * count, not this file):
 *   R1  the kernel is the 2-D Cauchy kernel 1/(z - y): Eq. (M2Lmat) is exactly
 *       its M2L with ME  phi(z) = sum_k m_k (z - x_s)^-(k+1),
 *       m_k = sum_i c_i (y_i - x_s)^k, and LE  phi(z) = sum_n l_n (z - x_t)^n.
 *   R2  p is the number of terms: n, k = 0 .. p-1.
 *   R3  interaction list of a box t at level l >= 2: the same-level children of
 *       the parent's neighbours (Chebyshev distance <= 1 between parents) that
 *       are not adjacent to t (Chebyshev distance >= 2).  Levels 0 and 1 are
 *       empty.  Corner contact counts as adjacent.  Order: parent offset ey
 *       major, ex minor, then child (cy major, cx minor).
 *   R4  periodic "paper-shape" lists wrap parent coordinates modulo 2^(l-1),
 *       so every box receives exactly 27 translations (Tables m2ltesla and
 *       m2lfermi count 27 * sum_l 4^l); the displacement is that of the
 *       periodic image.
 *   R5  points go to box floor(x * 2^l), clamped to 2^l - 1; box centres are
 *       geometric centres.
 *   R7  FGT: B_beta carries no (-1)^|beta| and the sum runs j = 1..N_B.
 *   R8  FGT: C_beta carries the factor (-1)^|beta| / beta! that Eq. (C_beta)
 *       omits.
 *   R9  FGT: delta = 2 sigma^2; tensor truncation alpha_i, beta_i < p.
 *   R12 adaptive tree (the paper describes only uniform subdivision): the
 *       root exists; an existing box holding more than q points is split
 *       while its level is below max_level; children holding no point are
 *       not created.  M2L on it runs over V-lists: the existing same-level
 *       children of the parent's colleagues (and of the parent) that are not
 *       adjacent to the target.  U/W/X lists are not part of the path.
 *   R13 far-field objective for gradients: J = sum_j w_j Re phi_far(z_j) at
 *       fixed evaluation points, phi_far(z) the L2P of the LE of z's leaf
 *       after M2L over V-lists at every level and L2L down; the topology
 *       (each point's leaf) is frozen when points move.
 *   R15 near field of a uniform tree at its finest level: a target takes the
 *       sources of its own box and of the (up to 8) adjacent boxes, the
 *       complement of the interaction lists of every level above; a source at
 *       exactly the target's position (the point itself) is skipped.
 *   R14 FGT Hermite evaluation on the grid (Sec. 4.2 takes the clusters of a
 *       target as given): a target takes every box within Chebyshev distance
 *       ncut of its own box, the neighbourhood the H2T uses (R9).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ------------------------------------------------------------------ */
/* small exact helpers                                                 */
/* ------------------------------------------------------------------ */

/* Binomial coefficients C(a, b), a <= 66, from Pascal's rule
 * C(a, b) = C(a-1, b-1) + C(a-1, b) in exact 64-bit integer arithmetic
 * (C(66, 33) ~ 7.2e18 < 2^64).  The conversion to double is exact up to
 * a = 56 and correctly rounded above; M2L uses a = n + k <= 2p - 2. */
#define PASCAL_MAX 66
static uint64_t pascal_tab[PASCAL_MAX + 1][PASCAL_MAX + 1];
static int pascal_ready = 0;

static void pascal_init(void)
{
    if (pascal_ready) return;
    for (int a = 0; a <= PASCAL_MAX; ++a) {
        for (int b = 0; b <= PASCAL_MAX; ++b) pascal_tab[a][b] = 0;
        pascal_tab[a][0] = 1;
        for (int b = 1; b <= a; ++b) pascal_tab[a][b] = pascal_tab[a - 1][b - 1] + pascal_tab[a - 1][b];
    }
    pascal_ready = 1;
}

static double binom(int a, int b)
{
    if (a > PASCAL_MAX) return NAN;
    if (b < 0 || b > a) return 0.0;
    pascal_init();
    return (double)pascal_tab[a][b];
}

static double factorial(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= (double)i;
    return f;
}

double orc_binom(int a, int b) { return binom(a, b); }

/* ------------------------------------------------------------------ */
/* quadtree geometry (Sec. 2.1, Fig. spatialDecomposition)             */
/* ------------------------------------------------------------------ */

static cplx box_centre(int level, int ix, int iy)
{
    double side = ldexp(1.0, -level);
    return ((double)ix + 0.5) * side + I * (((double)iy + 0.5) * side);
}

void orc_box_centre(int level, int ix, int iy, double* out /*re, im*/)
{
    cplx c = box_centre(level, ix, iy);
    out[0] = creal(c);
    out[1] = cimag(c);
}

/* box index of a point at a level (reading R5) */
static void point_box(int level, double x, double y, int* ix, int* iy)
{
    int n = 1 << level;
    int a = (int)floor(x * n), b = (int)floor(y * n);
    if (a < 0) a = 0;
    if (b < 0) b = 0;
    if (a > n - 1) a = n - 1;
    if (b > n - 1) b = n - 1;
    *ix = a;
    *iy = b;
}

/* ------------------------------------------------------------------ */
/* interaction list (Sec. 4.1 step 1; reading R3, R4)                   */
/* ------------------------------------------------------------------ */

/* Interaction list of target (tx, ty) at `level`.  Writes, for each entry,
 * the (wrapped) source box (sx, sy) and the source's image offset
 * (ox, oy) = image position - target position, in box units.  Returns the
 * number of entries (<= 27). */
int orc_interaction_list(int level, int tx, int ty, int periodic,
                         int* sx, int* sy, int* ox, int* oy)
{
    if (level < 2) return 0;
    int np = 1 << (level - 1);
    int px = tx >> 1, py = ty >> 1;
    int cnt = 0;
    for (int ey = -1; ey <= 1; ++ey) {
        for (int ex = -1; ex <= 1; ++ex) {
            int qx = px + ex, qy = py + ey; /* neighbour parent, unwrapped */
            if (!periodic && (qx < 0 || qy < 0 || qx >= np || qy >= np)) continue;
            for (int cy = 0; cy < 2; ++cy) {
                for (int cx = 0; cx < 2; ++cx) {
                    int ix = 2 * qx + cx, iy = 2 * qy + cy; /* image position */
                    int dx = ix - tx, dy = iy - ty;
                    int cheb = abs(dx) > abs(dy) ? abs(dx) : abs(dy);
                    if (cheb < 2) continue; /* adjacent (or itself): near field */
                    int n = 1 << level;
                    sx[cnt] = ((ix % n) + n) % n;
                    sy[cnt] = ((iy % n) + n) % n;
                    ox[cnt] = dx;
                    oy[cnt] = dy;
                    ++cnt;
                }
            }
        }
    }
    return cnt;
}

int64_t orc_list_count_level(int level, int periodic)
{
    int n = 1 << level;
    int64_t total = 0;
    int sx[27], sy[27], ox[27], oy[27];
    for (int ty = 0; ty < n; ++ty)
        for (int tx = 0; tx < n; ++tx)
            total += orc_interaction_list(level, tx, ty, periodic, sx, sy, ox, oy);
    return total;
}

/* ------------------------------------------------------------------ */
/* upward sweep (Sec. 2.1 stage 2) under reading R1                     */
/* ------------------------------------------------------------------ */

/* P2M of one box: m_k = sum_i c_i (y_i - x_c)^k, k < p. */
void orc_p2m_box(int64_t n, const double* xy, const double* c, double cx, double cy,
                 int p, double* m /* [p][2] */)
{
    cplx xc = cx + I * cy;
    cplx* acc = (cplx*)calloc((size_t)p, sizeof(cplx));
    for (int64_t i = 0; i < n; ++i) {
        cplx d = (xy[2 * i] + I * xy[2 * i + 1]) - xc;
        cplx pw = 1.0;
        for (int k = 0; k < p; ++k) {
            acc[k] += c[i] * pw;
            pw *= d;
        }
    }
    for (int k = 0; k < p; ++k) {
        m[2 * k] = creal(acc[k]);
        m[2 * k + 1] = cimag(acc[k]);
    }
    free(acc);
}

/* P2M for every box of a uniform level: M[b][k], b = iy * 2^l + ix. */
void orc_p2m_uniform(int level, int p, int64_t n, const double* xy, const double* c,
                     double* M /* [4^l][p][2] */)
{
    int nb = 1 << level;
    memset(M, 0, sizeof(double) * 2 * (size_t)p * (size_t)nb * (size_t)nb);
    for (int64_t i = 0; i < n; ++i) {
        int ix, iy;
        point_box(level, xy[2 * i], xy[2 * i + 1], &ix, &iy);
        cplx d = (xy[2 * i] + I * xy[2 * i + 1]) - box_centre(level, ix, iy);
        double* mb = M + 2 * (size_t)p * ((size_t)iy * nb + ix);
        cplx pw = 1.0;
        for (int k = 0; k < p; ++k) {
            cplx t = c[i] * pw;
            mb[2 * k] += creal(t);
            mb[2 * k + 1] += cimag(t);
            pw *= d;
        }
    }
}

/* M2M from the children at `child_level` to their parents:
 * M_j = sum_{k<=j} C(j,k) (x_c - x_P)^(j-k) m_k  (binomial shift of
 * (y - x_P)^j = ((y - x_c) + (x_c - x_P))^j). */
void orc_m2m_uniform(int child_level, int p, const double* Mc, double* Mp)
{
    int nc = 1 << child_level, npar = nc >> 1;
    memset(Mp, 0, sizeof(double) * 2 * (size_t)p * (size_t)npar * (size_t)npar);
    for (int iy = 0; iy < nc; ++iy) {
        for (int ix = 0; ix < nc; ++ix) {
            cplx z = box_centre(child_level, ix, iy) - box_centre(child_level - 1, ix >> 1, iy >> 1);
            const double* mc = Mc + 2 * (size_t)p * ((size_t)iy * nc + ix);
            double* mp = Mp + 2 * (size_t)p * ((size_t)(iy >> 1) * npar + (ix >> 1));
            cplx zp[128]; /* zp[e] = z^e */
            zp[0] = 1.0;
            for (int e = 1; e < p; ++e) zp[e] = zp[e - 1] * z;
            for (int j = 0; j < p; ++j) {
                cplx s = 0.0;
                for (int k = 0; k <= j; ++k) s += binom(j, k) * zp[j - k] * (mc[2 * k] + I * mc[2 * k + 1]);
                mp[2 * j] += creal(s);
                mp[2 * j + 1] += cimag(s);
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* M2L (Sec. 4.1 steps 2-3, Eq. M2Lmat)                                 */
/* ------------------------------------------------------------------ */

/* One translation: l_n += sum_k a_nk(d) m_k, d = x_t - x_s (target - source),
 * a_nk = (-1)^n C(n+k,k) d^(-(n+k+1)). */
void orc_m2l_pair(int p, double d_re, double d_im, const double* m, double* l)
{
    cplx d = d_re + I * d_im;
    cplx pw[256]; /* pw[j] = d^-j by repeated division, j < 2p */
    pw[0] = 1.0;
    for (int j = 1; j <= 2 * p - 1; ++j) pw[j] = pw[j - 1] / d;
    for (int n = 0; n < p; ++n) {
        cplx s = 0.0;
        double sign = (n % 2 == 0) ? 1.0 : -1.0;
        for (int k = 0; k < p; ++k) {
            cplx a = sign * binom(n + k, k) * pw[n + k + 1];
            s += a * (m[2 * k] + I * m[2 * k + 1]);
        }
        l[2 * n] += creal(s);
        l[2 * n + 1] += cimag(s);
    }
}

/* The p x p matrix a_nk(d), row-major [n][k][2]. */
void orc_m2l_matrix(int p, double d_re, double d_im, double* a)
{
    cplx d = d_re + I * d_im;
    cplx pw[256];
    pw[0] = 1.0;
    for (int j = 1; j <= 2 * p - 1; ++j) pw[j] = pw[j - 1] / d;
    for (int n = 0; n < p; ++n) {
        double sign = (n % 2 == 0) ? 1.0 : -1.0;
        for (int k = 0; k < p; ++k) {
            cplx v = sign * binom(n + k, k) * pw[n + k + 1];
            a[2 * (n * p + k)] = creal(v);
            a[2 * (n * p + k) + 1] = cimag(v);
        }
    }
}

/* M2L of a whole uniform level: for every target t, L_t = sum over the
 * interaction list of a(x_t - x_s) M_s (reduction by summation, in list
 * order).  L is overwritten.  Units are physical (unscaled). */
void orc_m2l_uniform(int level, int p, int periodic, const double* M, double* L)
{
    int n = 1 << level;
    double side = ldexp(1.0, -level);
    memset(L, 0, sizeof(double) * 2 * (size_t)p * (size_t)n * (size_t)n);
    int sx[27], sy[27], ox[27], oy[27];
    for (int ty = 0; ty < n; ++ty) {
        for (int tx = 0; tx < n; ++tx) {
            int cnt = orc_interaction_list(level, tx, ty, periodic, sx, sy, ox, oy);
            double* lt = L + 2 * (size_t)p * ((size_t)ty * n + tx);
            for (int e = 0; e < cnt; ++e) {
                /* d = x_t - x_s(image) = -(offset) * side */
                double dre = -(double)ox[e] * side, dim = -(double)oy[e] * side;
                const double* ms = M + 2 * (size_t)p * ((size_t)sy[e] * n + sx[e]);
                orc_m2l_pair(p, dre, dim, ms, lt);
            }
        }
    }
}

/* M2L restricted to a set of targets (for sampled checks at full size). */
void orc_m2l_uniform_targets(int level, int p, int periodic, const double* M,
                             int64_t ntarget, const int64_t* targets, double* Lout /*[ntarget][p][2]*/)
{
    int n = 1 << level;
    double side = ldexp(1.0, -level);
    int sx[27], sy[27], ox[27], oy[27];
    memset(Lout, 0, sizeof(double) * 2 * (size_t)p * (size_t)ntarget);
    for (int64_t i = 0; i < ntarget; ++i) {
        int tx = (int)(targets[i] % n), ty = (int)(targets[i] / n);
        int cnt = orc_interaction_list(level, tx, ty, periodic, sx, sy, ox, oy);
        for (int e = 0; e < cnt; ++e) {
            double dre = -(double)ox[e] * side, dim = -(double)oy[e] * side;
            const double* ms = M + 2 * (size_t)p * ((size_t)sy[e] * n + sx[e]);
            orc_m2l_pair(p, dre, dim, ms, Lout + 2 * (size_t)p * i);
        }
    }
}

/* Adjoint (plain transpose, no conjugation) of orc_m2l_uniform, by explicit
 * transposed loops: G_s[k] = sum_{t : s in IL(t)} sum_n a_nk(x_t - x_s) W_t[n]. */
void orc_m2l_adjoint_uniform(int level, int p, int periodic, const double* W, double* G)
{
    int n = 1 << level;
    double side = ldexp(1.0, -level);
    memset(G, 0, sizeof(double) * 2 * (size_t)p * (size_t)n * (size_t)n);
    int sx[27], sy[27], ox[27], oy[27];
    double* a = (double*)malloc(sizeof(double) * 2 * (size_t)p * (size_t)p);
    for (int ty = 0; ty < n; ++ty) {
        for (int tx = 0; tx < n; ++tx) {
            int cnt = orc_interaction_list(level, tx, ty, periodic, sx, sy, ox, oy);
            const double* wt = W + 2 * (size_t)p * ((size_t)ty * n + tx);
            for (int e = 0; e < cnt; ++e) {
                orc_m2l_matrix(p, -(double)ox[e] * side, -(double)oy[e] * side, a);
                double* gs = G + 2 * (size_t)p * ((size_t)sy[e] * n + sx[e]);
                for (int k = 0; k < p; ++k) {
                    cplx s = 0.0;
                    for (int nn = 0; nn < p; ++nn) {
                        cplx anks = a[2 * (nn * p + k)] + I * a[2 * (nn * p + k) + 1];
                        s += anks * (wt[2 * nn] + I * wt[2 * nn + 1]);
                    }
                    gs[2 * k] += creal(s);
                    gs[2 * k + 1] += cimag(s);
                }
            }
        }
    }
    free(a);
}

/* ------------------------------------------------------------------ */
/* far field and near field (Sec. 2.1 stages 4 and 5), for pins          */
/* ------------------------------------------------------------------ */

/* L2P: phi(z) = sum_n l_n (z - x_t)^n. */
void orc_l2p(int p, const double* l, double cx, double cy, int64_t nz, const double* z, double* phi)
{
    for (int64_t j = 0; j < nz; ++j) {
        cplx w = (z[2 * j] + I * z[2 * j + 1]) - (cx + I * cy);
        cplx s = 0.0, pw = 1.0;
        for (int n = 0; n < p; ++n) {
            s += (l[2 * n] + I * l[2 * n + 1]) * pw;
            pw *= w;
        }
        phi[2 * j] = creal(s);
        phi[2 * j + 1] = cimag(s);
    }
}

/* M2P: phi(z) = sum_k m_k (z - x_s)^-(k+1). */
void orc_m2p(int p, const double* m, double cx, double cy, int64_t nz, const double* z, double* phi)
{
    for (int64_t j = 0; j < nz; ++j) {
        cplx w = (z[2 * j] + I * z[2 * j + 1]) - (cx + I * cy);
        cplx s = 0.0, pw = 1.0 / w;
        for (int k = 0; k < p; ++k) {
            s += (m[2 * k] + I * m[2 * k + 1]) * pw;
            pw /= w;
        }
        phi[2 * j] = creal(s);
        phi[2 * j + 1] = cimag(s);
    }
}

/* Direct sum (Eq. n_body) with the Cauchy kernel: phi(z) = sum_i c_i / (z - y_i). */
void orc_direct(int64_t n, const double* xy, const double* c, int64_t nz, const double* z, double* phi)
{
    for (int64_t j = 0; j < nz; ++j) {
        cplx zj = z[2 * j] + I * z[2 * j + 1];
        cplx s = 0.0;
        for (int64_t i = 0; i < n; ++i) s += c[i] / (zj - (xy[2 * i] + I * xy[2 * i + 1]));
        phi[2 * j] = creal(s);
        phi[2 * j + 1] = cimag(s);
    }
}

/* Near field (Sec. 2.1 stage 5, Eq. n_body restricted, reading R15): for each
 * target z, the direct sum over the sources whose level-`level` box is its own
 * box or adjacent to it (Chebyshev distance <= 1), skipping sources at exactly
 * z's position:  phi(z) = sum_{i near z, y_i != z} c_i / (z - y_i). */
void orc_p2p_uniform(int level, int64_t n, const double* xy, const double* c, int64_t nz, const double* z,
                     double* phi)
{
    for (int64_t j = 0; j < nz; ++j) {
        int tx, ty;
        point_box(level, z[2 * j], z[2 * j + 1], &tx, &ty);
        cplx zj = z[2 * j] + I * z[2 * j + 1];
        cplx s = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            int sx, sy;
            point_box(level, xy[2 * i], xy[2 * i + 1], &sx, &sy);
            if (abs(sx - tx) > 1 || abs(sy - ty) > 1) continue;
            if (xy[2 * i] == z[2 * j] && xy[2 * i + 1] == z[2 * j + 1]) continue;
            s += c[i] / (zj - (xy[2 * i] + I * xy[2 * i + 1]));
        }
        phi[2 * j] = creal(s);
        phi[2 * j + 1] = cimag(s);
    }
}

/* L2L: re-centre an LE from x_P to x_c: l'_j = sum_{n>=j} C(n,j) (x_c - x_P)^(n-j) l_n. */
void orc_l2l(int p, const double* lp, double dre, double dim, double* lc)
{
    cplx z = dre + I * dim; /* x_c - x_P */
    cplx zp[128];
    zp[0] = 1.0;
    for (int e = 1; e < p; ++e) zp[e] = zp[e - 1] * z;
    for (int j = 0; j < p; ++j) {
        cplx s = 0.0;
        for (int n = j; n < p; ++n) s += binom(n, j) * zp[n - j] * (lp[2 * n] + I * lp[2 * n + 1]);
        lc[2 * j] = creal(s);
        lc[2 * j + 1] = cimag(s);
    }
}

/* ------------------------------------------------------------------ */
/* Fast Gauss transform (Sec. 2.2)                                      */
/* ------------------------------------------------------------------ */

/* Hermite functions h_n(t) = e^{-t^2} H_n(t), n = 0..nmax-1, by the
 * three-term recurrence of the (physicists') Hermite polynomials
 * H_{n+1} = 2t H_n - 2n H_{n-1}. */
void orc_hermite_functions(int nmax, double t, double* h)
{
    if (nmax <= 0) return;
    h[0] = exp(-t * t);
    if (nmax > 1) h[1] = 2.0 * t * h[0];
    for (int n = 1; n + 1 < nmax; ++n) h[n + 1] = 2.0 * t * h[n] - 2.0 * (double)n * h[n - 1];
}

/* Direct Gauss transform (Eq. dgt): G(y) = sum_i q_i exp(-|x_i - y|^2 / (2 sigma^2)). */
void orc_fgt_direct(int64_t n, const double* x, const double* q, double sigma,
                    int64_t ny, const double* y, double* G)
{
    for (int64_t j = 0; j < ny; ++j) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double dx = x[2 * i] - y[2 * j], dy = x[2 * i + 1] - y[2 * j + 1];
            s += q[i] * exp(-(dx * dx + dy * dy) / (2.0 * sigma * sigma));
        }
        G[j] = s;
    }
}

/* Hermite coefficients about s_B (Eq. A_alpha):
 * A[a1][a2] = (1/(a1! a2!)) sum_j q_j t1^a1 t2^a2,  t = (x_j - s_B)/(sqrt(2) sigma). */
void orc_fgt_p2h(int64_t n, const double* x, const double* q, double sbx, double sby,
                 double sigma, int p, double* A /* [p][p] */)
{
    double sc = sqrt(2.0) * sigma;
    memset(A, 0, sizeof(double) * (size_t)p * (size_t)p);
    double* f = (double*)malloc(sizeof(double) * (size_t)p);
    double* w1 = (double*)malloc(sizeof(double) * (size_t)p);
    double* w2 = (double*)malloc(sizeof(double) * (size_t)p);
    for (int k = 0; k < p; ++k) f[k] = factorial(k);
    for (int64_t j = 0; j < n; ++j) {
        double t1 = (x[2 * j] - sbx) / sc, t2 = (x[2 * j + 1] - sby) / sc;
        w1[0] = 1.0;
        w2[0] = 1.0;
        for (int k = 1; k < p; ++k) {
            w1[k] = w1[k - 1] * t1;
            w2[k] = w2[k - 1] * t2;
        }
        for (int a1 = 0; a1 < p; ++a1)
            for (int a2 = 0; a2 < p; ++a2) A[a1 * p + a2] += q[j] * w1[a1] * w2[a2] / (f[a1] * f[a2]);
    }
    free(f);
    free(w1);
    free(w2);
}

/* Hermite-series evaluation (Eq. hermite): G(y) = sum_alpha A_alpha h_alpha((y - s_B)/(sqrt(2) sigma)). */
void orc_fgt_hermite_eval(int p, const double* A, double sbx, double sby, double sigma,
                          int64_t ny, const double* y, double* G)
{
    double sc = sqrt(2.0) * sigma;
    double* h1 = (double*)malloc(sizeof(double) * (size_t)p);
    double* h2 = (double*)malloc(sizeof(double) * (size_t)p);
    for (int64_t j = 0; j < ny; ++j) {
        orc_hermite_functions(p, (y[2 * j] - sbx) / sc, h1);
        orc_hermite_functions(p, (y[2 * j + 1] - sby) / sc, h2);
        double s = 0.0;
        for (int a1 = 0; a1 < p; ++a1)
            for (int a2 = 0; a2 < p; ++a2) s += A[a1 * p + a2] * h1[a1] * h2[a2];
        G[j] = s;
    }
    free(h1);
    free(h2);
}

/* Taylor coefficients about t_C (Eq. B_beta, reading R7):
 * B[b1][b2] = sum_j q_j h_b1(s1) h_b2(s2) / (b1! b2!),  s = (x_j - t_C)/(sqrt(2) sigma). */
void orc_fgt_p2t(int64_t n, const double* x, const double* q, double tcx, double tcy,
                 double sigma, int p, double* B)
{
    double sc = sqrt(2.0) * sigma;
    double* h1 = (double*)malloc(sizeof(double) * (size_t)p);
    double* h2 = (double*)malloc(sizeof(double) * (size_t)p);
    memset(B, 0, sizeof(double) * (size_t)p * (size_t)p);
    for (int64_t j = 0; j < n; ++j) {
        orc_hermite_functions(p, (x[2 * j] - tcx) / sc, h1);
        orc_hermite_functions(p, (x[2 * j + 1] - tcy) / sc, h2);
        for (int b1 = 0; b1 < p; ++b1)
            for (int b2 = 0; b2 < p; ++b2)
                B[b1 * p + b2] += q[j] * h1[b1] * h2[b2] / (factorial(b1) * factorial(b2));
    }
    free(h1);
    free(h2);
}

/* Taylor-series evaluation (Eq. taylor): G(y) = sum_beta B_beta ((y - t_C)/(sqrt(2) sigma))^beta. */
void orc_fgt_taylor_eval(int p, const double* B, double tcx, double tcy, double sigma,
                         int64_t ny, const double* y, double* G)
{
    double sc = sqrt(2.0) * sigma;
    for (int64_t j = 0; j < ny; ++j) {
        double t1 = (y[2 * j] - tcx) / sc, t2 = (y[2 * j + 1] - tcy) / sc;
        double s = 0.0;
        for (int b1 = 0; b1 < p; ++b1)
            for (int b2 = 0; b2 < p; ++b2) s += B[b1 * p + b2] * pow(t1, b1) * pow(t2, b2);
        G[j] = s;
    }
}

/* One Hermite-to-Taylor translation (Eq. C_beta with reading R8):
 * C[b1][b2] += ((-1)^(b1+b2) / (b1! b2!)) sum_{a1,a2} A[a1][a2] h_{a1+b1}(u1) h_{a2+b2}(u2),
 * u = (t_C - s_B)/(sqrt(2) sigma). */
void orc_fgt_h2t_pair(int p, const double* A, double u1, double u2, double* C)
{
    double* h1 = (double*)malloc(sizeof(double) * (size_t)(2 * p));
    double* h2 = (double*)malloc(sizeof(double) * (size_t)(2 * p));
    orc_hermite_functions(2 * p - 1, u1, h1);
    orc_hermite_functions(2 * p - 1, u2, h2);
    for (int b1 = 0; b1 < p; ++b1) {
        for (int b2 = 0; b2 < p; ++b2) {
            double s = 0.0;
            for (int a1 = 0; a1 < p; ++a1)
                for (int a2 = 0; a2 < p; ++a2) s += A[a1 * p + a2] * h1[a1 + b1] * h2[a2 + b2];
            double sign = ((b1 + b2) % 2 == 0) ? 1.0 : -1.0;
            C[b1 * p + b2] += sign * s / (factorial(b1) * factorial(b2));
        }
    }
    free(h1);
    free(h2);
}

/* H2T over a uniform grid of 2^g x 2^g boxes on [0,1)^2: every target box t
 * receives the translations of every source box s with
 * max(|sx - tx|, |sy - ty|) <= n_cut.  A, C are [4^g][p][p], box b = iy*2^g+ix.
 * C is overwritten. */
void orc_fgt_h2t_grid(int g, int ncut, int p, double sigma, const double* A, double* C)
{
    int n = 1 << g;
    double side = ldexp(1.0, -g), sc = sqrt(2.0) * sigma;
    memset(C, 0, sizeof(double) * (size_t)p * (size_t)p * (size_t)n * (size_t)n);
    for (int ty = 0; ty < n; ++ty) {
        for (int tx = 0; tx < n; ++tx) {
            for (int sy = ty - ncut; sy <= ty + ncut; ++sy) {
                for (int sx = tx - ncut; sx <= tx + ncut; ++sx) {
                    if (sx < 0 || sy < 0 || sx >= n || sy >= n) continue;
                    double u1 = ((double)(tx - sx) * side) / sc;
                    double u2 = ((double)(ty - sy) * side) / sc;
                    orc_fgt_h2t_pair(p, A + (size_t)p * p * ((size_t)sy * n + sx), u1, u2,
                                     C + (size_t)p * p * ((size_t)ty * n + tx));
                }
            }
        }
    }
}

/* H2T for a subset of target boxes (sampled checks). */
void orc_fgt_h2t_targets(int g, int ncut, int p, double sigma, const double* A,
                         int64_t ntarget, const int64_t* targets, double* Cout)
{
    int n = 1 << g;
    double side = ldexp(1.0, -g), sc = sqrt(2.0) * sigma;
    memset(Cout, 0, sizeof(double) * (size_t)p * (size_t)p * (size_t)ntarget);
    for (int64_t i = 0; i < ntarget; ++i) {
        int tx = (int)(targets[i] % n), ty = (int)(targets[i] / n);
        for (int sy = ty - ncut; sy <= ty + ncut; ++sy) {
            for (int sx = tx - ncut; sx <= tx + ncut; ++sx) {
                if (sx < 0 || sy < 0 || sx >= n || sy >= n) continue;
                double u1 = ((double)(tx - sx) * side) / sc;
                double u2 = ((double)(ty - sy) * side) / sc;
                orc_fgt_h2t_pair(p, A + (size_t)p * p * ((size_t)sy * n + sx), u1, u2,
                                 Cout + (size_t)p * p * i);
            }
        }
    }
}

/* Hermite-series evaluation on the uniform FGT grid (Eq. hermite, reading R14):
 * each target y takes every source box B whose Chebyshev distance, in boxes,
 * from y's own box is at most ncut (boxes outside the grid do not exist),
 *   G(y) = sum_B sum_{a1,a2 < p} A_B[a1][a2] h_a1((y1 - sB1)/(sqrt2 sigma)) h_a2((y2 - sB2)/(sqrt2 sigma)),
 * s_B the centre of B.  Source boxes in row-major order (sy outer, sx inner). */
void orc_fgt_hermite_eval_grid(int g, int ncut, int p, double sigma, const double* A, int64_t ny,
                               const double* y, double* G)
{
    int nb = 1 << g;
    double side = ldexp(1.0, -g);
    for (int64_t j = 0; j < ny; ++j) {
        int tx, ty;
        point_box(g, y[2 * j], y[2 * j + 1], &tx, &ty);
        double acc = 0.0;
        for (int sy = ty - ncut; sy <= ty + ncut; ++sy) {
            for (int sx = tx - ncut; sx <= tx + ncut; ++sx) {
                if (sx < 0 || sy < 0 || sx >= nb || sy >= nb) continue;
                double v = 0.0;
                orc_fgt_hermite_eval(p, A + (size_t)p * p * ((size_t)sy * nb + sx), ((double)sx + 0.5) * side,
                                     ((double)sy + 0.5) * side, sigma, 1, y + 2 * j, &v);
                acc += v;
            }
        }
        G[j] = acc;
    }
}

/* P2H for every box of the uniform FGT grid (Eq. A_alpha per box). */
void orc_fgt_p2h_grid(int g, int p, double sigma, int64_t n, const double* x, const double* q, double* A)
{
    int nb = 1 << g;
    double side = ldexp(1.0, -g), sc = sqrt(2.0) * sigma;
    memset(A, 0, sizeof(double) * (size_t)p * (size_t)p * (size_t)nb * (size_t)nb);
    double* f = (double*)malloc(sizeof(double) * (size_t)p);
    double* w1 = (double*)malloc(sizeof(double) * (size_t)p);
    double* w2 = (double*)malloc(sizeof(double) * (size_t)p);
    for (int k = 0; k < p; ++k) f[k] = factorial(k);
    for (int64_t j = 0; j < n; ++j) {
        int ix, iy;
        point_box(g, x[2 * j], x[2 * j + 1], &ix, &iy);
        double t1 = (x[2 * j] - ((double)ix + 0.5) * side) / sc;
        double t2 = (x[2 * j + 1] - ((double)iy + 0.5) * side) / sc;
        double* Ab = A + (size_t)p * p * ((size_t)iy * nb + ix);
        w1[0] = 1.0;
        w2[0] = 1.0;
        for (int k = 1; k < p; ++k) {
            w1[k] = w1[k - 1] * t1;
            w2[k] = w2[k - 1] * t2;
        }
        for (int a1 = 0; a1 < p; ++a1)
            for (int a2 = 0; a2 < p; ++a2) Ab[a1 * p + a2] += q[j] * w1[a1] * w2[a2] / (f[a1] * f[a2]);
    }
    free(f);
    free(w1);
    free(w2);
}

/* ------------------------------------------------------------------ */
/* adaptive quadtree, V-lists and the far field on it (reading R12)     */
/* ------------------------------------------------------------------ */

/* Boxes of all levels 0..L are numbered level by level: box b of level l is
 * entry (4^l - 1)/3 + b of a per-tree array, b = iy * 2^l + ix. */
static int64_t level_offset(int l) { return (((int64_t)1 << (2 * l)) - 1) / 3; }

int64_t orc_level_offset(int l) { return level_offset(l); }

/* Adaptive tree over levels 0..max_level (reading R12): the root exists; an
 * existing box of level l < max_level holding more than q points is split,
 * and each of its four children that holds at least one point exists.
 * exists[] has level_offset(max_level + 1) entries.  Returns the deepest
 * level that has an existing box. */
int orc_adaptive_tree(int64_t n, const double* xy, int q, int max_level, uint8_t* exists)
{
    memset(exists, 0, (size_t)level_offset(max_level + 1));
    exists[0] = 1;
    int depth = 0;
    int64_t* cnt_parent = NULL;
    for (int l = 0; l <= max_level; ++l) {
        int side = 1 << l;
        int64_t* cnt = (int64_t*)calloc((size_t)side * side, sizeof(int64_t));
        for (int64_t i = 0; i < n; ++i) {
            int ix, iy;
            point_box(l, xy[2 * i], xy[2 * i + 1], &ix, &iy);
            cnt[(int64_t)iy * side + ix] += 1;
        }
        if (l > 0) {
            int pside = side / 2;
            for (int iy = 0; iy < side; ++iy)
                for (int ix = 0; ix < side; ++ix) {
                    int64_t pb = (int64_t)(iy / 2) * pside + ix / 2;
                    int parent_split = exists[level_offset(l - 1) + pb] && cnt_parent[pb] > q;
                    if (parent_split && cnt[(int64_t)iy * side + ix] > 0) {
                        exists[level_offset(l) + (int64_t)iy * side + ix] = 1;
                        depth = l;
                    }
                }
        }
        free(cnt_parent);
        cnt_parent = cnt;
    }
    free(cnt_parent);
    return depth;
}

/* V-list of target (tx, ty) at `level` of an adaptive tree: the existing
 * boxes of the same level that are children of the target's parent or of
 * one of the parent's colleagues (same-level boxes at Chebyshev distance 1
 * from the parent) and are not adjacent to the target.  Empty when the
 * target does not exist.  Output as orc_interaction_list (no periodicity). */
int orc_vlist(int level, int tx, int ty, const uint8_t* exists, int* sx, int* sy, int* ox, int* oy)
{
    if (level < 2) return 0;
    int side = 1 << level, pside = side / 2;
    if (!exists[level_offset(level) + (int64_t)ty * side + tx]) return 0;
    int ptx = tx / 2, pty = ty / 2;
    int cnt = 0;
    for (int qy = pty - 1; qy <= pty + 1; ++qy) {
        for (int qx = ptx - 1; qx <= ptx + 1; ++qx) {
            if (qx < 0 || qy < 0 || qx >= pside || qy >= pside) continue;
            if (!exists[level_offset(level - 1) + (int64_t)qy * pside + qx]) continue; /* not a colleague */
            for (int cy = 0; cy < 2; ++cy) {
                for (int cx = 0; cx < 2; ++cx) {
                    int ix = 2 * qx + cx, iy = 2 * qy + cy;
                    if (!exists[level_offset(level) + (int64_t)iy * side + ix]) continue;
                    int dx = ix - tx, dy = iy - ty;
                    int adx = dx < 0 ? -dx : dx, ady = dy < 0 ? -dy : dy;
                    if ((adx > ady ? adx : ady) <= 1) continue; /* adjacent: U-list, near field */
                    sx[cnt] = ix;
                    sy[cnt] = iy;
                    ox[cnt] = dx;
                    oy[cnt] = dy;
                    ++cnt;
                }
            }
        }
    }
    return cnt;
}

int64_t orc_vlist_count_level(int level, const uint8_t* exists)
{
    int side = 1 << level;
    int64_t total = 0;
    int sx[27], sy[27], ox[27], oy[27];
    for (int ty = 0; ty < side; ++ty)
        for (int tx = 0; tx < side; ++tx) total += orc_vlist(level, tx, ty, exists, sx, sy, ox, oy);
    return total;
}

/* M2L of one level of an adaptive tree over the V-lists (Sec. 4.1 steps 2-3,
 * Eq. M2Lmat): L_t = sum_{s in V(t)} a(x_t - x_s) M_s for existing t; zero
 * for boxes that do not exist.  M, L: [4^level][p] complex, physical units. */
void orc_m2l_adaptive(int level, int p, const uint8_t* exists, const double* M, double* L)
{
    int side = 1 << level;
    double h = ldexp(1.0, -level);
    memset(L, 0, sizeof(double) * 2 * (size_t)p * (size_t)side * (size_t)side);
    int sx[27], sy[27], ox[27], oy[27];
    for (int ty = 0; ty < side; ++ty)
        for (int tx = 0; tx < side; ++tx) {
            int cnt = orc_vlist(level, tx, ty, exists, sx, sy, ox, oy);
            double* lt = L + 2 * (size_t)p * ((size_t)ty * side + tx);
            for (int e = 0; e < cnt; ++e)
                orc_m2l_pair(p, -(double)ox[e] * h, -(double)oy[e] * h,
                             M + 2 * (size_t)p * ((size_t)sy[e] * side + sx[e]), lt);
        }
}

/* Plain transpose of orc_m2l_adaptive by explicit transposed loops:
 * G_s[k] = sum_{t : s in V(t)} sum_n a_nk(x_t - x_s) W_t[n]. */
void orc_m2l_adjoint_adaptive(int level, int p, const uint8_t* exists, const double* W, double* G)
{
    int side = 1 << level;
    double h = ldexp(1.0, -level);
    memset(G, 0, sizeof(double) * 2 * (size_t)p * (size_t)side * (size_t)side);
    int sx[27], sy[27], ox[27], oy[27];
    double* a = (double*)malloc(sizeof(double) * 2 * (size_t)p * (size_t)p);
    for (int ty = 0; ty < side; ++ty)
        for (int tx = 0; tx < side; ++tx) {
            int cnt = orc_vlist(level, tx, ty, exists, sx, sy, ox, oy);
            const double* wt = W + 2 * (size_t)p * ((size_t)ty * side + tx);
            for (int e = 0; e < cnt; ++e) {
                orc_m2l_matrix(p, -(double)ox[e] * h, -(double)oy[e] * h, a);
                double* gs = G + 2 * (size_t)p * ((size_t)sy[e] * side + sx[e]);
                for (int k = 0; k < p; ++k) {
                    cplx s = 0.0;
                    for (int nn = 0; nn < p; ++nn)
                        s += (a[2 * (nn * p + k)] + I * a[2 * (nn * p + k) + 1]) * (wt[2 * nn] + I * wt[2 * nn + 1]);
                    gs[2 * k] += creal(s);
                    gs[2 * k + 1] += cimag(s);
                }
            }
        }
    free(a);
}

/* M2L contributions of a few source boxes only: for every existing target t
 * of the level within Chebyshev distance 3 of a listed source s, adds
 * a(x_t - x_s) M_s to L_t when s is in V(t).  M: [nsrc][p] complex (the
 * sources' MEs), L: [4^level][p] complex (accumulated). */
void orc_m2l_adaptive_from_sources(int level, int p, const uint8_t* exists, int64_t nsrc, const int64_t* src,
                                   const double* M, double* L)
{
    int side = 1 << level;
    double h = ldexp(1.0, -level);
    int sx[27], sy[27], ox[27], oy[27];
    for (int64_t i = 0; i < nsrc; ++i) {
        int bx = (int)(src[i] % side), by = (int)(src[i] / side);
        for (int ty = by - 3; ty <= by + 3; ++ty)
            for (int tx = bx - 3; tx <= bx + 3; ++tx) {
                if (tx < 0 || ty < 0 || tx >= side || ty >= side) continue;
                int cnt = orc_vlist(level, tx, ty, exists, sx, sy, ox, oy);
                for (int e = 0; e < cnt; ++e) {
                    if (sx[e] != bx || sy[e] != by) continue;
                    orc_m2l_pair(p, -(double)ox[e] * h, -(double)oy[e] * h, M + 2 * (size_t)p * i,
                                 L + 2 * (size_t)p * ((size_t)ty * side + tx));
                }
            }
    }
}

/* P2M with a given box per point (frozen topology): for every point i with
 * box[i] >= 0, M[box[i]][k] += c_i (y_i - x_box)^k.  M: [4^level][p] complex,
 * accumulated. */
void orc_p2m_assigned(int level, int p, int64_t n, const double* xy, const double* c, const int64_t* box, double* M)
{
    int side = 1 << level;
    for (int64_t i = 0; i < n; ++i) {
        if (box[i] < 0) continue;
        int bx = (int)(box[i] % side), by = (int)(box[i] / side);
        cplx d = (xy[2 * i] + I * xy[2 * i + 1]) - box_centre(level, bx, by);
        cplx pw = c[i];
        double* m = M + 2 * (size_t)p * (size_t)box[i];
        for (int k = 0; k < p; ++k) {
            m[2 * k] += creal(pw);
            m[2 * k + 1] += cimag(pw);
            pw *= d;
        }
    }
}

/* L2L from level child_level - 1 to the existing boxes of child_level:
 * Lc[child] += l2l(Lp[parent]) (Sec. 2.1 stage 3, downward sweep). */
void orc_l2l_level(int child_level, int p, const uint8_t* exists, const double* Lp, double* Lc)
{
    int side = 1 << child_level, pside = side / 2;
    double* tmp = (double*)malloc(sizeof(double) * 2 * (size_t)p);
    for (int iy = 0; iy < side; ++iy)
        for (int ix = 0; ix < side; ++ix) {
            if (!exists[level_offset(child_level) + (int64_t)iy * side + ix]) continue;
            cplx shift = box_centre(child_level, ix, iy) - box_centre(child_level - 1, ix / 2, iy / 2);
            orc_l2l(p, Lp + 2 * (size_t)p * ((size_t)(iy / 2) * pside + ix / 2), creal(shift), cimag(shift), tmp);
            double* lc = Lc + 2 * (size_t)p * ((size_t)iy * side + ix);
            for (int k = 0; k < 2 * p; ++k) lc[k] += tmp[k];
        }
    free(tmp);
}
