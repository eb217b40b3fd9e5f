/*
 * rid_oracle.c -- plain FP64 CPU oracle for the Reinforced Dynamics (RiD)
 * biased / restrained Langevin MD step over many walkers.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code, header or table
 * with the CUDA library; the two meet only through the seeded input arrays.
 *
 * Everything is double precision, written for checkability rather than speed:
 * one function per step of the method, in the order the method applies them.
 * The only single-precision arithmetic is the Lennard-Jones inclusion test
 * r^2 < rc^2, which is an integer decision and is therefore taken in the same
 * precision as the GPU kernel (FP32, r^2 formed with two fused multiply-adds
 * in a fixed order; build with -ffp-contract=off so nothing else is fused).
 *
 * What each part follows (RiD-kit paper, arXiv 2408.14070):
 *   - mean force F(s) = grad_s A(s), A = -kT ln p(s)               (Box 2)
 *   - bias = inverted PMF predicted by the ensemble, applied only where the
 *     model deviation is low; trust_lvl_1 / trust_lvl_2 are the lower / upper
 *     uncertainty bounds                                  (Sec. "Development
 *     of the protocol"; Sec. "Overall workflow setting")
 *   - model deviation = spread of the ensemble members' predictions
 *                                                        (Sec. "Training phase")
 *   - ensemble MLP with `neurons` hidden widths and optional residual
 *     connections between equal-width layers             (Sec. "Training phase")
 *   - torsion CVs, periodic over 2 pi, and distance CVs between two beads
 *     (not periodic; the MLP takes (s, 0) for them)     (Sec. "CV selection")
 *   - restrained MD labelling: harmonic restraints with force constants
 *     `kappas`, mean force estimated by the spring force   (Sec. "Labeling
 *     phase", restrained method; Sec. "Development of the protocol")
 * Readings where the paper is silent (switching function, force field forms,
 * integrator, random numbers) are stated at each function.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel     */
/* random numbers: as easy as 1, 2, 3", SC'11).  Counter = (c0,c1,c2,c3),   */
/* key = (k0,k1).  Each of the 10 rounds multiplies c0 and c2 by the two    */
/* round multipliers, mixes the high halves with the other two words and    */
/* the key, and then bumps the key by the two Weyl constants.               */
/* ------------------------------------------------------------------------ */
static const uint32_t PHILOX_M0 = 0xD2511F53u, PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u, PHILOX_W1 = 0xBB67AE85u;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void orc_philox_batch(int64_t n, const uint32_t* ctr, uint64_t seed, uint32_t* out)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t i = 0; i < n; ++i) orc_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

/* Three standard normals for one (bead, walker, step, stream) counter.
 * Reading (the paper names no integrator noise): counter = (bead, walker,
 * step, stream), key = (seed lo, seed hi); each 32-bit word x becomes
 * u = (x + 1/2) 2^-32 in (0, 1); Box-Muller on (u0, u1) gives xi_x, xi_y and
 * on (u2, u3) gives xi_z (its sine partner is dropped). */
void orc_normals3(uint64_t seed, uint32_t bead, uint32_t walker, uint32_t step,
                  uint32_t stream, double xi[3])
{
    uint32_t ctr[4] = {bead, walker, step, stream}, key[2], o[4];
    key[0] = (uint32_t)seed; key[1] = (uint32_t)(seed >> 32);
    orc_philox4x32_10(ctr, key, o);
    double u[4];
    for (int k = 0; k < 4; ++k) u[k] = ((double)o[k] + 0.5) * 0x1p-32;
    double r0 = sqrt(-2.0 * log(u[0])), r1 = sqrt(-2.0 * log(u[2]));
    xi[0] = r0 * cos(2.0 * ORC_PI * u[1]);
    xi[1] = r0 * sin(2.0 * ORC_PI * u[1]);
    xi[2] = r1 * cos(2.0 * ORC_PI * u[3]);
}

void orc_normals_batch(int64_t n, const uint32_t* bws /* [n][4] bead,walker,step,stream */,
                       uint64_t seed, double* out /* [n][3] */)
{
    for (int64_t i = 0; i < n; ++i)
        orc_normals3(seed, bws[4 * i], bws[4 * i + 1], bws[4 * i + 2], bws[4 * i + 3], out + 3 * i);
}

/* ------------------------------------------------------------------------ */
/* System and ensemble descriptions                                          */
/* ------------------------------------------------------------------------ */
typedef struct {
    int n;                      /* beads */
    double mass, kT, dt, gamma;
    uint64_t seed;
    double kb, r0, ka, theta0;  /* bonds, angles */
    const double* dk;           /* [n-3][3] dihedral amplitudes k_1..k_3 */
    const double* dd;           /* [n-3][3] dihedral phases delta_1..delta_3 */
    double lj_eps, lj_sig, lj_rc;
    int n_cv;
    const int32_t* cv;          /* [C][4] bead indices of each CV: a torsion of four beads, or the
                                   distance between the first two when the last two are -1 */
    int output_freq;
} orc_sys;

/* CV kind: the distance between beads cv[j][0] and cv[j][1] when cv[j][2] < 0. */
static int cv_is_distance(const int32_t* cv, int j) { return cv[4 * j + 2] < 0; }

typedef struct {
    int M, D, L, H, resnet;
    double e0, e1;              /* trust_lvl_1, trust_lvl_2 */
    const double* w;            /* [M][P] packed, see orc_model_param_count */
} orc_ens;

static int64_t model_param_count(int D, int L, int H)
{
    return (int64_t)H * D + H + (int64_t)(L - 1) * ((int64_t)H * H + H) + H + 1;
}

int64_t orc_model_param_count(int D, int L, int H) { return model_param_count(D, L, H); }

/* ------------------------------------------------------------------------ */
/* Vector helpers                                                            */
/* ------------------------------------------------------------------------ */
static inline void vsub(const double* a, const double* b, double* o)
{ o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static inline double vdot(const double* a, const double* b)
{ return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static inline void vcross(const double* a, const double* b, double* o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static inline double vnorm(const double* a) { return sqrt(vdot(a, a)); }

/* Periodic difference onto [-pi, pi): d - 2 pi floor(d / 2 pi + 1/2).
 * Reading: ties at +-pi go to -pi (half-open interval). */
static double wrap_pi(double d)
{
    return d - 2.0 * ORC_PI * floor(d / (2.0 * ORC_PI) + 0.5);
}
double orc_wrap_pi(double d) { return wrap_pi(d); }

/* Restraint offset of CV j from its centre: wrapped for a torsion, plain
 * for a distance. */
static double cv_offset(const int32_t* cv, int j, double s, double s0)
{
    return (cv && cv[4 * j + 2] < 0) ? s - s0 : wrap_pi(s - s0);
}

/* ------------------------------------------------------------------------ */
/* Torsion angle of four points and its gradient.                            */
/* Convention (IUPAC): phi = atan2(|b2| b1.(b2 x b3), (b1 x b2).(b2 x b3))   */
/* with b1 = p1-p0, b2 = p2-p1, b3 = p3-p2; cis = 0, trans = +-pi, mapped    */
/* onto [-pi, pi).  Gradient in the form of Blondel & Karplus (J. Comput.   */
/* Chem. 17, 1132 (1996)), written with F = p0-p1, G = p1-p2, H = p3-p2,     */
/* A = F x G, B = H x G.                                                     */
/* ------------------------------------------------------------------------ */
double orc_dihedral(const double* p /* [4][3] */, double* grad /* [4][3] or NULL */)
{
    double b1[3], b2[3], b3[3], m[3], n[3];
    vsub(p + 3, p + 0, b1);
    vsub(p + 6, p + 3, b2);
    vsub(p + 9, p + 6, b3);
    vcross(b1, b2, m);
    vcross(b2, b3, n);
    double lb2 = vnorm(b2);
    double phi = atan2(lb2 * vdot(b1, n), vdot(m, n));
    if (phi >= ORC_PI) phi -= 2.0 * ORC_PI;
    if (grad) {
        double F[3], G[3], H[3], A[3], B[3];
        vsub(p + 0, p + 3, F);
        vsub(p + 3, p + 6, G);
        vsub(p + 9, p + 6, H);
        vcross(F, G, A);
        vcross(H, G, B);
        double A2 = vdot(A, A), B2 = vdot(B, B), lG = vnorm(G);
        double fg = vdot(F, G), hg = vdot(H, G);
        for (int k = 0; k < 3; ++k) {
            double a = A[k], b = B[k];
            grad[0 + k] = -lG / A2 * a;
            grad[9 + k] = lG / B2 * b;
            grad[3 + k] = lG / A2 * a + fg / (A2 * lG) * a - hg / (B2 * lG) * b;
            grad[6 + k] = -lG / B2 * b - fg / (A2 * lG) * a + hg / (B2 * lG) * b;
        }
    }
    return phi;
}

/* ------------------------------------------------------------------------ */
/* Force field of the bead chain (stand-in for the paper's GROMACS force     */
/* field; forms are a reading: harmonic terms k/2 d^2, three-term cosine    */
/* dihedrals, Lennard-Jones truncated at rc with the potential shifted to   */
/* zero at rc and the force truncated, pairs |i-j| >= 3 only).              */
/* Returns the potential; adds -grad U into f (if f != NULL).               */
/* terms[0..3] (if non-NULL) = bond, angle, dihedral, LJ energies.          */
/* ------------------------------------------------------------------------ */

/* Pair inclusion decision, taken in the precision of the kernel: FP32
 * differences and r^2 = fma(dz, dz, fma(dy, dy, dx dx)) with correctly rounded
 * fused multiply-adds (C99 fmaf), so both sides decide identically. */
static int lj_included(const double* xi, const double* xj, float rc2f)
{
    float dx = (float)xj[0] - (float)xi[0];
    float dy = (float)xj[1] - (float)xi[1];
    float dz = (float)xj[2] - (float)xi[2];
    float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    return r2 < rc2f;
}

double orc_ff(const orc_sys* S, const double* x, double* f, double* terms)
{
    const int N = S->n;
    double Ub = 0, Ua = 0, Ud = 0, Ul = 0;
    /* bonds (i, i+1) */
    for (int i = 0; i + 1 < N; ++i) {
        double d[3];
        vsub(x + 3 * (i + 1), x + 3 * i, d);
        double r = vnorm(d), dr = r - S->r0;
        Ub += 0.5 * S->kb * dr * dr;
        if (f) {
            double c = S->kb * dr / r;   /* dU/dr / r */
            for (int k = 0; k < 3; ++k) { f[3 * i + k] += c * d[k]; f[3 * (i + 1) + k] -= c * d[k]; }
        }
    }
    /* angles (i, i+1, i+2), vertex i+1 */
    for (int i = 0; i + 2 < N; ++i) {
        double a[3], b[3], axb[3];
        vsub(x + 3 * i, x + 3 * (i + 1), a);
        vsub(x + 3 * (i + 2), x + 3 * (i + 1), b);
        vcross(a, b, axb);
        double la = vnorm(a), lb = vnorm(b);
        double th = atan2(vnorm(axb), vdot(a, b));
        double dth = th - S->theta0;
        Ua += 0.5 * S->ka * dth * dth;
        if (f) {
            double dU = S->ka * dth, c = cos(th), s = sin(th);
            for (int k = 0; k < 3; ++k) {
                double ah = a[k] / la, bh = b[k] / lb;
                double ga = (c * ah - bh) / (la * s);   /* d theta / d a */
                double gb = (c * bh - ah) / (lb * s);   /* d theta / d b */
                f[3 * i + k] -= dU * ga;
                f[3 * (i + 2) + k] -= dU * gb;
                f[3 * (i + 1) + k] += dU * (ga + gb);
            }
        }
    }
    /* dihedrals (i .. i+3) */
    for (int i = 0; i + 3 < N; ++i) {
        double g[12];
        double phi = orc_dihedral(x + 3 * i, f ? g : NULL);
        double dU = 0;
        for (int nn = 1; nn <= 3; ++nn) {
            double kn = S->dk[3 * i + nn - 1], dn = S->dd[3 * i + nn - 1];
            Ud += kn * (1.0 + cos(nn * phi - dn));
            dU -= nn * kn * sin(nn * phi - dn);
        }
        if (f)
            for (int q = 0; q < 12; ++q) f[3 * i + q] -= dU * g[q];
    }
    /* Lennard-Jones, non-excluded pairs */
    const float rc2f = (float)(S->lj_rc * S->lj_rc);
    const double s2 = S->lj_sig * S->lj_sig, rc2 = S->lj_rc * S->lj_rc;
    const double src6 = s2 * s2 * s2 / (rc2 * rc2 * rc2);
    const double Urc = 4.0 * S->lj_eps * (src6 * src6 - src6);
    for (int i = 0; i < N; ++i)
        for (int j = i + 3; j < N; ++j) {
            if (!lj_included(x + 3 * i, x + 3 * j, rc2f)) continue;
            double d[3];
            vsub(x + 3 * j, x + 3 * i, d);
            double r2 = vdot(d, d);
            double sr2 = s2 / r2, sr6 = sr2 * sr2 * sr2;
            Ul += 4.0 * S->lj_eps * (sr6 * sr6 - sr6) - Urc;
            if (f) {
                double c = 24.0 * S->lj_eps * (2.0 * sr6 * sr6 - sr6) / r2;
                for (int k = 0; k < 3; ++k) { f[3 * i + k] -= c * d[k]; f[3 * j + k] += c * d[k]; }
            }
        }
    if (terms) { terms[0] = Ub; terms[1] = Ua; terms[2] = Ud; terms[3] = Ul; }
    return Ub + Ua + Ud + Ul;
}

/* Pairs that pass the LJ inclusion test, from FP32 positions.  Writes up to
 * cap (i, j) pairs with i < j in row-major order; returns the count. */
int64_t orc_lj_pairs(int n, const float* xf /* [n][3] */, double rc, int64_t cap, int32_t* out)
{
    const float rc2f = (float)(rc * rc);
    int64_t c = 0;
    for (int i = 0; i < n; ++i)
        for (int j = i + 3; j < n; ++j) {
            double xi[3] = {xf[3 * i], xf[3 * i + 1], xf[3 * i + 2]};
            double xj[3] = {xf[3 * j], xf[3 * j + 1], xf[3 * j + 2]};
            if (lj_included(xi, xj, rc2f)) {
                if (c < cap) { out[2 * c] = i; out[2 * c + 1] = j; }
                ++c;
            }
        }
    return c;
}

/* ------------------------------------------------------------------------ */
/* CVs (Sec. "CV selection": torsions and distances): s_j = torsion of beads  */
/* cv[j][0..3], or s_j = |x_b - x_a| for a distance CV (a, b, -1, -1);       */
/* J[j] = d s_j / d x on its 4 slots (a distance uses slots 0 and 1:          */
/* -(x_b - x_a)/s and +(x_b - x_a)/s; slots 2, 3 are zero).                   */
/* ------------------------------------------------------------------------ */
static void cvs_eval(const orc_sys* S, const double* x, double* s, double* J /* [C][12] */)
{
    for (int j = 0; j < S->n_cv; ++j) {
        if (cv_is_distance(S->cv, j)) {
            const int a = S->cv[4 * j], b = S->cv[4 * j + 1];
            double r[3];
            vsub(x + 3 * b, x + 3 * a, r);
            const double d = vnorm(r);
            s[j] = d;
            if (J) {
                double* g = J + 12 * j;
                for (int k = 0; k < 3; ++k) { g[k] = -r[k] / d; g[3 + k] = r[k] / d; g[6 + k] = 0; g[9 + k] = 0; }
            }
            continue;
        }
        double p[12];
        for (int a = 0; a < 4; ++a)
            for (int k = 0; k < 3; ++k) p[3 * a + k] = x[3 * S->cv[4 * j + a] + k];
        s[j] = orc_dihedral(p, J ? J + 12 * j : NULL);
    }
}

/* ------------------------------------------------------------------------ */
/* One ensemble member: input u = (cos s_0, sin s_0, cos s_1, sin s_1, ...),  */
/* hidden layers h_l = tanh(W_l h_{l-1} + b_l) (plus h_{l-1} for l >= 2 when */
/* resnet), output A = w_out . h_L + b_out.  Then reverse-mode input        */
/* gradient: g_L = w_out, g_{l-1} = W_l^T (g_l * (1 - tanh^2)) (+ g_l for a   */
/* residual layer), dA/du = g_0.                                            */
/* Packed parameters: W1[H][D], b1[H], (W_l[H][H], b_l[H]) l=2..L, w_out[H], */
/* b_out.                                                                   */
/* ------------------------------------------------------------------------ */
static void mlp_eval(const orc_ens* E, int m, const double* u, double* A_out, double* dAdu)
{
    const int D = E->D, L = E->L, H = E->H;
    const double* w = E->w + (int64_t)m * model_param_count(D, L, H);
    double* t = (double*)malloc(sizeof(double) * (size_t)L * H);   /* tanh(z_l) */
    double* h = (double*)malloc(sizeof(double) * (size_t)(L + 1) * H);
    double* g = (double*)malloc(sizeof(double) * (size_t)(H > D ? H : D));
    double* gp = (double*)malloc(sizeof(double) * (size_t)(H > D ? H : D));
    const double* Wl[64];
    const double* bl[64];
    const double* p = w;
    for (int l = 0; l < L; ++l) {
        int fin = l == 0 ? D : H;
        Wl[l] = p; p += (int64_t)H * fin;
        bl[l] = p; p += H;
    }
    const double* wout = p;
    const double bout = p[H];
    /* forward */
    const double* prev = u;
    for (int l = 0; l < L; ++l) {
        int fin = l == 0 ? D : H;
        for (int o = 0; o < H; ++o) {
            double z = bl[l][o];
            for (int i = 0; i < fin; ++i) z += Wl[l][(int64_t)o * fin + i] * prev[i];
            t[l * H + o] = tanh(z);
            h[l * H + o] = t[l * H + o] + ((E->resnet && l > 0) ? prev[o] : 0.0);
        }
        prev = h + l * H;
    }
    double A = bout;
    for (int o = 0; o < H; ++o) A += wout[o] * prev[o];
    if (A_out) *A_out = A;
    /* backward */
    for (int o = 0; o < H; ++o) g[o] = wout[o];
    for (int l = L - 1; l >= 0; --l) {
        int fin = l == 0 ? D : H;
        for (int i = 0; i < fin; ++i) {
            double acc = 0;
            for (int o = 0; o < H; ++o) {
                double tz = t[l * H + o];
                acc += Wl[l][(int64_t)o * fin + i] * g[o] * (1.0 - tz * tz);
            }
            if (E->resnet && l > 0) acc += g[i];
            gp[i] = acc;
        }
        memcpy(g, gp, sizeof(double) * (size_t)fin);
    }
    if (dAdu) memcpy(dAdu, g, sizeof(double) * (size_t)D);
    free(t); free(h); free(g); free(gp);
}

/* Flat-argument wrapper for tests: A_i(u) and dA_i/du for one member. */
void orc_mlp(int M, int D, int L, int H, int resnet, const double* w, int m,
             const double* u, double* A, double* dAdu)
{
    orc_ens E = {M, D, L, H, resnet, 0, 0, w};
    mlp_eval(&E, m, u, A, dAdu);
}

/* Switching factor sigma(eps).  Reading (the paper only says: bias where the
 * model deviation is low, with trust_lvl_1 / trust_lvl_2 as the lower / upper
 * bounds): the cosine switch of the original RiD work, 1 below e0, 0 at or
 * above e1, (1 + cos(pi (eps - e0)/(e1 - e0)))/2 in between. */
static double switch_sigma(double eps, double e0, double e1)
{
    if (eps < e0) return 1.0;
    if (eps >= e1) return 0.0;
    return 0.5 * (1.0 + cos(ORC_PI * (eps - e0) / (e1 - e0)));
}
double orc_switch(double eps, double e0, double e1) { return switch_sigma(eps, e0, e1); }

/* Ensemble at CV point s: member gradients dA_i/ds, mean force
 * Fbar = (1/M) sum_i dA_i/ds, deviation eps = sqrt((1/M) sum_i |dA_i/ds - Fbar|^2)
 * (population, Euclidean over the C CV components), switched CV force
 * F_s = sigma(eps) Fbar (the bias potential is -Abar, so its force on s is
 * +grad Abar).  Abar = mean member value. */
/* MLP input of CV j (reading: the paper feeds periodic CVs through their   */
/* cosine and sine; a distance CV, not periodic, enters as (s_j, 0)), and    */
/* dA/ds_j from dA/du by the chain rule through that map.                   */
static void ensemble_eval(const orc_ens* E, int C, const double* s, const int32_t* cv, double* Fs,
                          double* eps_out, double* Abar_out, double* sig_out, double* gradA /* [M][C] or NULL */)
{
    const int M = E->M, D = E->D;
    double* u = (double*)malloc(sizeof(double) * (size_t)D);
    double* du = (double*)malloc(sizeof(double) * (size_t)D);
    double* gA = (double*)malloc(sizeof(double) * (size_t)M * C);
    for (int j = 0; j < C; ++j) {
        if (cv && cv_is_distance(cv, j)) { u[2 * j] = s[j]; u[2 * j + 1] = 0.0; }
        else { u[2 * j] = cos(s[j]); u[2 * j + 1] = sin(s[j]); }
    }
    double Abar = 0;
    for (int m = 0; m < M; ++m) {
        double A;
        mlp_eval(E, m, u, &A, du);
        Abar += A / M;
        for (int j = 0; j < C; ++j)
            gA[m * C + j] = (cv && cv_is_distance(cv, j)) ? du[2 * j]
                                                          : -sin(s[j]) * du[2 * j] + cos(s[j]) * du[2 * j + 1];
    }
    double e2 = 0;
    for (int j = 0; j < C; ++j) {
        double fb = 0;
        for (int m = 0; m < M; ++m) fb += gA[m * C + j];
        Fs[j] = fb / M;
    }
    for (int m = 0; m < M; ++m)
        for (int j = 0; j < C; ++j) { double d = gA[m * C + j] - Fs[j]; e2 += d * d; }
    double eps = sqrt(e2 / M);
    double sig = switch_sigma(eps, E->e0, E->e1);
    for (int j = 0; j < C; ++j) Fs[j] *= sig;
    if (eps_out) *eps_out = eps;
    if (Abar_out) *Abar_out = Abar;
    if (sig_out) *sig_out = sig;
    if (gradA) memcpy(gradA, gA, sizeof(double) * (size_t)M * C);
    free(u); free(du); free(gA);
}

/* ------------------------------------------------------------------------ */
/* Total force at x: force field + CV force chain-ruled to the beads.       */
/* mode 0: no CV force; 1: ensemble bias; 2: harmonic restraint with         */
/* centres s0 and constants kappa: F_s = -kappa (wrap(s - s0)).             */
/* Outputs s (C), eps, Abar (mode 1), U_ff.                                 */
/* ------------------------------------------------------------------------ */
typedef struct {
    int mode;
    const orc_ens* E;
    const double* s0;
    const double* kappa;
} orc_bias;

static double total_force(const orc_sys* S, const orc_bias* B, const double* x, double* f,
                          double* s, double* eps, double* Abar, double* Urest)
{
    const int N = S->n, C = S->n_cv;
    memset(f, 0, sizeof(double) * 3 * (size_t)N);
    double U = orc_ff(S, x, f, NULL);
    double* J = (double*)malloc(sizeof(double) * 12 * (size_t)(C > 0 ? C : 1));
    double* Fs = (double*)malloc(sizeof(double) * (size_t)(C > 0 ? C : 1));
    cvs_eval(S, x, s, J);
    double e = 0, ab = 0, ur = 0;
    if (B->mode == 1 && B->E) {
        ensemble_eval(B->E, C, s, S->cv, Fs, &e, &ab, NULL, NULL);
    } else if (B->mode == 2) {
        for (int j = 0; j < C; ++j) {
            double d = cv_offset(S->cv, j, s[j], B->s0[j]);
            Fs[j] = -B->kappa[j] * d;
            ur += 0.5 * B->kappa[j] * d * d;
        }
    } else {
        for (int j = 0; j < C; ++j) Fs[j] = 0;
    }
    for (int j = 0; j < C; ++j)
        for (int a = 0; a < 4; ++a) {
            int at = S->cv[4 * j + a];
            if (at < 0) continue;
            for (int k = 0; k < 3; ++k) f[3 * at + k] += Fs[j] * J[12 * j + 3 * a + k];
        }
    if (eps) *eps = e;
    if (Abar) *Abar = ab;
    if (Urest) *Urest = ur;
    free(J); free(Fs);
    return U;
}

/* ------------------------------------------------------------------------ */
/* BAOAB Langevin step (reading: the paper names no integrator; Leimkuhler & */
/* Matthews' BAOAB with one force evaluation per step):                      */
/*   B: v += dt/2 f/m; A: x += dt/2 v; O: v = c1 v + c2 xi;                  */
/*   A: x += dt/2 v; f = F(x); B: v += dt/2 f/m,                             */
/* c1 = exp(-gamma dt), c2 = sqrt((1 - c1^2) kT/m), xi from Philox stream 0  */
/* at counter (bead, walker, step, 0).  gamma = 0 is velocity Verlet.        */
/* The force evaluation is left to the caller (split as pre / post).         */
/* ------------------------------------------------------------------------ */
static void baoab_pre(int n, int dim, double* x, double* v, const double* f, double m,
                      double dt, double gamma, double kT, uint64_t seed, uint32_t walker, uint32_t step)
{
    const double c1 = exp(-gamma * dt), c2 = sqrt((1.0 - c1 * c1) * kT / m);
    for (int i = 0; i < n; ++i) {
        double xi[3] = {0, 0, 0};
        if (gamma > 0) orc_normals3(seed, (uint32_t)i, walker, step, 0u, xi);
        for (int k = 0; k < dim; ++k) {
            double* vv = v + dim * i + k;
            double* xx = x + dim * i + k;
            *vv += 0.5 * dt * f[dim * i + k] / m;
            *xx += 0.5 * dt * *vv;
            *vv = c1 * *vv + c2 * xi[k];
            *xx += 0.5 * dt * *vv;
        }
    }
}

static void baoab_post(int n, int dim, double* v, const double* f, double m, double dt)
{
    for (int i = 0; i < n * dim; ++i) v[i] += 0.5 * dt * f[i] / m;
}

/* Maxwell-Boltzmann velocities from Philox stream 1 at counter
 * (bead, walker, step0, 1). */
static void mb_velocities(int n, double* v, double m, double kT, uint64_t seed, uint32_t walker, uint32_t step0)
{
    const double sd = sqrt(kT / m);
    for (int i = 0; i < n; ++i) {
        double xi[3];
        orc_normals3(seed, (uint32_t)i, walker, step0, 1u, xi);
        for (int k = 0; k < 3; ++k) v[3 * i + k] = sd * xi[k];
    }
}

/* ------------------------------------------------------------------------ */
/* Restrained-MD mean-force statistics (Sec. "Labeling phase", restrained):  */
/* for every CV the restraint displacement d = wrap(s - s0) is sampled after */
/* each step past n_equil; MF = -kappa mean(d); standard error from B equal */
/* blocks, SE = kappa std_{ddof=1}(block means)/sqrt(B); std = population    */
/* std of kappa d.  Sample k of K goes to block floor(k B / K).             */
/* ------------------------------------------------------------------------ */
typedef struct {
    int C, B;
    int64_t K;
    double* sum;    /* [C] */
    double* sum2;   /* [C] */
    double* bsum;   /* [C][B] */
} orc_stats;

static void stats_init(orc_stats* st, int C, int B, int64_t K)
{
    st->C = C; st->B = B; st->K = K;
    st->sum = (double*)calloc((size_t)C, sizeof(double));
    st->sum2 = (double*)calloc((size_t)C, sizeof(double));
    st->bsum = (double*)calloc((size_t)C * B, sizeof(double));
}
static void stats_free(orc_stats* st) { free(st->sum); free(st->sum2); free(st->bsum); }

static void stats_add(orc_stats* st, int64_t k, const double* d)
{
    int b = (int)((k * st->B) / st->K);
    for (int j = 0; j < st->C; ++j) {
        st->sum[j] += d[j];
        st->sum2[j] += d[j] * d[j];
        st->bsum[j * st->B + b] += d[j];
    }
}

static void stats_finish(const orc_stats* st, const double* kappa, double* mf, double* se, double* sd)
{
    const int B = st->B;
    const int64_t K = st->K;
    for (int j = 0; j < st->C; ++j) {
        double mean = st->sum[j] / (double)K;
        double var = st->sum2[j] / (double)K - mean * mean;
        if (var < 0) var = 0;
        double bm_mean = 0, bm[4096];
        for (int b = 0; b < B; ++b) {
            int64_t lo = (b * K + B - 1) / B, hi = ((b + 1) * K + B - 1) / B;  /* k with floor(kB/K) == b */
            bm[b] = st->bsum[j * B + b] / (double)(hi - lo);
            bm_mean += bm[b] / B;
        }
        double ss = 0;
        for (int b = 0; b < B; ++b) ss += (bm[b] - bm_mean) * (bm[b] - bm_mean);
        mf[j] = -kappa[j] * mean;
        se[j] = kappa[j] * sqrt(ss / (B - 1) / B);
        sd[j] = kappa[j] * sqrt(var);
    }
}

/* ------------------------------------------------------------------------ */
/* Drivers                                                                   */
/* ------------------------------------------------------------------------ */
typedef struct {
    const orc_sys* S;
    const orc_ens* E;
    int W;
    const float* x0;      /* [W][N][3] */
    const float* v0;      /* [W][N][3] or NULL */
    uint64_t step0;
    int64_t n_steps;
    /* explore */
    float* cv_out;        /* [W][T][C] */
    float* eps_out;       /* [W][T] */
    double* energy_out;   /* [W][T][3]: U_ff, -Abar, kinetic; or NULL */
    /* label */
    int label;
    const double* s0;     /* [W][C] */
    const double* kappa;  /* [W][C] */
    int64_t n_equil;
    int n_blocks;
    double* mf_out; double* se_out; double* sd_out;   /* [W][C] */
    /* both */
    double* x_out;        /* [W][N][3] or NULL */
    double* v_out;        /* [W][N][3] or NULL */
    int n_threads;
    int next;             /* work counter */
    pthread_mutex_t mu;
} run_ctx;

static void run_walker(run_ctx* R, int w)
{
    const orc_sys* S = R->S;
    const int N = S->n, C = S->n_cv;
    double* x = (double*)malloc(sizeof(double) * 3 * (size_t)N);
    double* v = (double*)malloc(sizeof(double) * 3 * (size_t)N);
    double* f = (double*)malloc(sizeof(double) * 3 * (size_t)N);
    double* s = (double*)malloc(sizeof(double) * (size_t)(C > 0 ? C : 1));
    double* d = (double*)malloc(sizeof(double) * (size_t)(C > 0 ? C : 1));
    for (int i = 0; i < 3 * N; ++i) x[i] = R->x0[(int64_t)w * 3 * N + i];
    if (R->v0) for (int i = 0; i < 3 * N; ++i) v[i] = R->v0[(int64_t)w * 3 * N + i];
    else mb_velocities(N, v, S->mass, S->kT, S->seed, (uint32_t)w, (uint32_t)R->step0);
    orc_bias B = {0, NULL, NULL, NULL};
    if (R->label) { B.mode = 2; B.s0 = R->s0 + (int64_t)w * C; B.kappa = R->kappa + (int64_t)w * C; }
    else if (R->E) { B.mode = 1; B.E = R->E; }
    orc_stats st;
    memset(&st, 0, sizeof(st));
    if (R->label) stats_init(&st, C, R->n_blocks, R->n_steps - R->n_equil);
    double eps, Abar;
    total_force(S, &B, x, f, s, &eps, &Abar, NULL);
    const int64_t T = S->output_freq > 0 ? R->n_steps / S->output_freq : 0;
    for (int64_t t = 0; t < R->n_steps; ++t) {
        uint32_t step = (uint32_t)(R->step0 + (uint64_t)t);
        baoab_pre(N, 3, x, v, f, S->mass, S->dt, S->gamma, S->kT, S->seed, (uint32_t)w, step);
        double Uff = total_force(S, &B, x, f, s, &eps, &Abar, NULL);
        baoab_post(N, 3, v, f, S->mass, S->dt);
        if (R->label && t >= R->n_equil) {
            for (int j = 0; j < C; ++j) d[j] = cv_offset(S->cv, j, s[j], B.s0[j]);
            stats_add(&st, t - R->n_equil, d);
        }
        if (!R->label && S->output_freq > 0 && (t + 1) % S->output_freq == 0) {
            int64_t slot = (t + 1) / S->output_freq - 1;
            if (slot < T) {
                if (R->cv_out) for (int j = 0; j < C; ++j) R->cv_out[((int64_t)w * T + slot) * C + j] = (float)s[j];
                if (R->eps_out) R->eps_out[(int64_t)w * T + slot] = (float)eps;
                if (R->energy_out) {
                    double ke = 0;
                    for (int i = 0; i < 3 * N; ++i) ke += 0.5 * S->mass * v[i] * v[i];
                    double* e = R->energy_out + ((int64_t)w * T + slot) * 3;
                    e[0] = Uff; e[1] = (B.mode == 1) ? -Abar : 0.0; e[2] = ke;
                }
            }
        }
    }
    if (R->label) {
        stats_finish(&st, B.kappa, R->mf_out + (int64_t)w * C, R->se_out + (int64_t)w * C,
                     R->sd_out + (int64_t)w * C);
        stats_free(&st);
    }
    if (R->x_out) for (int i = 0; i < 3 * N; ++i) R->x_out[(int64_t)w * 3 * N + i] = x[i];
    if (R->v_out) for (int i = 0; i < 3 * N; ++i) R->v_out[(int64_t)w * 3 * N + i] = v[i];
    free(x); free(v); free(f); free(s); free(d);
}

static void* run_thread(void* arg)
{
    run_ctx* R = (run_ctx*)arg;
    for (;;) {
        pthread_mutex_lock(&R->mu);
        int w = R->next++;
        pthread_mutex_unlock(&R->mu);
        if (w >= R->W) break;
        run_walker(R, w);
    }
    return NULL;
}

static int run_all(run_ctx* R)
{
    int nt = R->n_threads;
    if (nt <= 0) nt = (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (nt < 1) nt = 1;
    if (nt > R->W) nt = R->W;
    R->next = 0;
    pthread_mutex_init(&R->mu, NULL);
    pthread_t th[512];
    if (nt > 512) nt = 512;
    for (int i = 0; i < nt; ++i) pthread_create(&th[i], NULL, run_thread, R);
    for (int i = 0; i < nt; ++i) pthread_join(th[i], NULL);
    pthread_mutex_destroy(&R->mu);
    return nt;
}

/* Flat-argument system constructor used by all entry points below. */
static void make_sys(orc_sys* S, int n, double mass, double kT, double dt, double gamma, uint64_t seed,
                     double kb, double r0, double ka, double th0, const double* dk, const double* dd,
                     double eps, double sig, double rc, int n_cv, const int32_t* cv, int output_freq)
{
    S->n = n; S->mass = mass; S->kT = kT; S->dt = dt; S->gamma = gamma; S->seed = seed;
    S->kb = kb; S->r0 = r0; S->ka = ka; S->theta0 = th0; S->dk = dk; S->dd = dd;
    S->lj_eps = eps; S->lj_sig = sig; S->lj_rc = rc; S->n_cv = n_cv; S->cv = cv;
    S->output_freq = output_freq;
}

/* sys_d = {mass, kT, dt, gamma, kb, r0, ka, theta0, lj_eps, lj_sig, lj_rc}
 * sys_i = {n_beads, n_cv, output_freq}                                     */
#define SYS_ARGS const double* sys_d, const int32_t* sys_i, uint64_t seed, const double* dk, \
                 const double* dd, const int32_t* cv
#define SYS_MAKE(S) make_sys(&(S), sys_i[0], sys_d[0], sys_d[1], sys_d[2], sys_d[3], seed, sys_d[4], \
                             sys_d[5], sys_d[6], sys_d[7], dk, dd, sys_d[8], sys_d[9], sys_d[10], \
                             sys_i[1], cv, sys_i[2])
/* ens_i = {M, D, L, H, resnet}, ens_d = {e0, e1}                           */

/* Force-field energy / forces and CV values / Jacobians at one configuration. */
double orc_eval_ff(SYS_ARGS, const double* x, double* f, double* terms)
{
    orc_sys S; SYS_MAKE(S);
    if (f) memset(f, 0, sizeof(double) * 3 * (size_t)S.n);
    return orc_ff(&S, x, f, terms);
}

void orc_eval_cvs(SYS_ARGS, const double* x, double* s, double* J)
{
    orc_sys S; SYS_MAKE(S);
    cvs_eval(&S, x, s, J);
}

/* Ensemble quantities at CV point s: F_s (switched), eps, Abar, sigma, dA_i/ds.
 * cv: the system's [C][4] CV atoms (for the CV kinds), or NULL for torsions only. */
void orc_eval_ensemble(const int32_t* ens_i, const double* ens_d, const double* w, int C, const int32_t* cv,
                       const double* s, double* Fs, double* out3 /* eps, Abar, sigma */, double* gradA)
{
    orc_ens E = {ens_i[0], ens_i[1], ens_i[2], ens_i[3], ens_i[4], ens_d[0], ens_d[1], w};
    ensemble_eval(&E, C, s, cv, Fs, &out3[0], &out3[1], &out3[2], gradA);
}

/* Total force at one configuration: mode 0 none, 1 ensemble bias, 2 restraint.
 * out4 = {U_ff, eps, Abar, U_restraint}. */
void orc_eval_total(SYS_ARGS, const int32_t* ens_i, const double* ens_d, const double* w,
                    int mode, const double* s0, const double* kappa,
                    const double* x, double* f, double* s, double* out4)
{
    orc_sys S; SYS_MAKE(S);
    orc_ens E;
    if (ens_i) { E.M = ens_i[0]; E.D = ens_i[1]; E.L = ens_i[2]; E.H = ens_i[3]; E.resnet = ens_i[4];
                 E.e0 = ens_d[0]; E.e1 = ens_d[1]; E.w = w; }
    orc_bias B = {mode, ens_i ? &E : NULL, s0, kappa};
    out4[0] = total_force(&S, &B, x, f, s, &out4[1], &out4[2], &out4[3]);
}

/* Biased exploration of W walkers (ens_i == NULL: unbiased MD).  Returns the
 * number of threads used. */
int orc_explore(SYS_ARGS, const int32_t* ens_i, const double* ens_d, const double* w,
                int W, const float* x0, const float* v0, uint64_t step0, int64_t n_steps,
                float* cv_out, float* eps_out, double* energy_out, double* x_out, double* v_out,
                int n_threads)
{
    orc_sys S; SYS_MAKE(S);
    orc_ens E;
    if (ens_i) { E.M = ens_i[0]; E.D = ens_i[1]; E.L = ens_i[2]; E.H = ens_i[3]; E.resnet = ens_i[4];
                 E.e0 = ens_d[0]; E.e1 = ens_d[1]; E.w = w; }
    run_ctx R;
    memset(&R, 0, sizeof(R));
    R.S = &S; R.E = ens_i ? &E : NULL; R.W = W; R.x0 = x0; R.v0 = v0; R.step0 = step0;
    R.n_steps = n_steps; R.cv_out = cv_out; R.eps_out = eps_out; R.energy_out = energy_out;
    R.x_out = x_out; R.v_out = v_out; R.n_threads = n_threads;
    return run_all(&R);
}

/* Restrained labelling runs, one per starting configuration. */
int orc_label(SYS_ARGS, int R_, const float* x0, const float* v0, const double* s0, const double* kappa,
              uint64_t step0, int64_t n_steps, int64_t n_equil, int n_blocks,
              double* mf, double* se, double* sd, double* x_out, double* v_out, int n_threads)
{
    orc_sys S; SYS_MAKE(S);
    if (n_blocks < 2 || n_blocks > 4096 || n_steps - n_equil < n_blocks) return -1;
    run_ctx R;
    memset(&R, 0, sizeof(R));
    R.S = &S; R.W = R_; R.x0 = x0; R.v0 = v0; R.step0 = step0; R.n_steps = n_steps;
    R.label = 1; R.s0 = s0; R.kappa = kappa; R.n_equil = n_equil; R.n_blocks = n_blocks;
    R.mf_out = mf; R.se_out = se; R.sd_out = sd; R.x_out = x_out; R.v_out = v_out;
    R.n_threads = n_threads;
    return run_all(&R);
}

/* ------------------------------------------------------------------------ */
/* Constrained-MD labels (Sec. "Labeling phase", constrained method; Box 5:   */
/* distance CVs only).  Reading: each distance CV r_j = |x_a - x_b| (pairs   */
/* of distinct beads, no bead in two pairs, equal masses) is held at d0_j by */
/* BAOAB with SHAKE / RATTLE projections:                                    */
/*   B  v += dt/2 f/m, project v;                                           */
/*   A  x_old = x, x += dt/2 v, SHAKE x (and v), project v;                 */
/*   O  v = c1 v + c2 xi (the noise of the unconstrained step), project v;  */
/*   A  as above;  f = F_ff(x);  B  v += dt/2 f/m, project v.               */
/* SHAKE for one distance: x_a -= lam r_old, x_b += lam r_old with the      */
/* smaller root of |r' - 2 lam r_old| = d0; v gets the same change / h.     */
/* Projection of v: the relative velocity along u = (x_a - x_b)/d0 is       */
/* removed symmetrically.                                                    */
/* Mean force on r_j after each step past n_equil (thermodynamic integration */
/* along the distance, with the Jacobian r^2 of the spherical shell):        */
/*   F_j = dU/dr - 2 kT / d0 = -(f_a - f_b) . u / 2 - 2 kT / d0,             */
/* which equals -<lambda> of the rigid-constraint force; MF = <F>, SE from  */
/* n_blocks blocks, std = population std of F.                              */
/* ------------------------------------------------------------------------ */
static void cons_shake(int C, const int32_t* pr, const double* d0, const double* xo, double* x, double* v, double h)
{
    for (int j = 0; j < C; ++j) {
        const int a = pr[2 * j], b = pr[2 * j + 1];
        double ro[3], rp[3];
        for (int k = 0; k < 3; ++k) {
            ro[k] = xo[3 * a + k] - xo[3 * b + k];
            rp[k] = x[3 * a + k] - x[3 * b + k];
        }
        const double ro2 = ro[0] * ro[0] + ro[1] * ro[1] + ro[2] * ro[2];
        const double rpo = rp[0] * ro[0] + rp[1] * ro[1] + rp[2] * ro[2];
        const double rp2 = rp[0] * rp[0] + rp[1] * rp[1] + rp[2] * rp[2];
        const double dd = rpo * rpo - ro2 * (rp2 - d0[j] * d0[j]);
        const double lam = (rp2 - d0[j] * d0[j]) / (2.0 * (rpo + sqrt(dd > 0 ? dd : 0)));
        for (int k = 0; k < 3; ++k) {
            x[3 * a + k] -= lam * ro[k];
            x[3 * b + k] += lam * ro[k];
            v[3 * a + k] -= lam * ro[k] / h;
            v[3 * b + k] += lam * ro[k] / h;
        }
    }
}

static void cons_project_v(int C, const int32_t* pr, const double* x, double* v)
{
    for (int j = 0; j < C; ++j) {
        const int a = pr[2 * j], b = pr[2 * j + 1];
        double u[3], r = 0, w = 0;
        for (int k = 0; k < 3; ++k) {
            u[k] = x[3 * a + k] - x[3 * b + k];
            r += u[k] * u[k];
        }
        r = sqrt(r);
        for (int k = 0; k < 3; ++k) {
            u[k] /= r;
            w += (v[3 * a + k] - v[3 * b + k]) * u[k];
        }
        w *= 0.5;
        for (int k = 0; k < 3; ++k) {
            v[3 * a + k] -= w * u[k];
            v[3 * b + k] += w * u[k];
        }
    }
}

int orc_label_constrained(SYS_ARGS, int R_, const float* x0, const float* v0, int C, const int32_t* pairs,
                          const double* d0 /* [R][C] */, uint64_t step0, int64_t n_steps, int64_t n_equil,
                          int n_blocks, double* mf, double* se, double* sd, double* x_out, double* v_out)
{
    orc_sys S; SYS_MAKE(S);
    const int N = S.n;
    if (n_blocks < 2 || n_blocks > 4096 || n_steps - n_equil < n_blocks || C < 1) return -1;
    const double m = S.mass, dt = S.dt;
    const double c1 = exp(-S.gamma * dt), c2 = sqrt((1.0 - c1 * c1) * S.kT / m);
    double* x = (double*)malloc(sizeof(double) * 3 * (size_t)N);
    double* xo = (double*)malloc(sizeof(double) * 3 * (size_t)N);
    double* v = (double*)malloc(sizeof(double) * 3 * (size_t)N);
    double* f = (double*)malloc(sizeof(double) * 3 * (size_t)N);
    double* smp = (double*)malloc(sizeof(double) * (size_t)C);
    double* one = (double*)malloc(sizeof(double) * (size_t)C);
    for (int j = 0; j < C; ++j) one[j] = 1.0;
    for (int r = 0; r < R_; ++r) {
        const double* dr = d0 + (size_t)r * C;
        for (int i = 0; i < 3 * N; ++i) x[i] = x0[(size_t)r * 3 * N + i];
        /* start on the constraint surface: each pair moved symmetrically along its own axis */
        for (int j = 0; j < C; ++j) {
            const int a = pairs[2 * j], b = pairs[2 * j + 1];
            double u[3], len = 0, c[3];
            for (int k = 0; k < 3; ++k) {
                u[k] = x[3 * a + k] - x[3 * b + k];
                c[k] = 0.5 * (x[3 * a + k] + x[3 * b + k]);
                len += u[k] * u[k];
            }
            len = sqrt(len);
            for (int k = 0; k < 3; ++k) {
                x[3 * a + k] = c[k] + 0.5 * dr[j] * u[k] / len;
                x[3 * b + k] = c[k] - 0.5 * dr[j] * u[k] / len;
            }
        }
        if (v0) for (int i = 0; i < 3 * N; ++i) v[i] = v0[(size_t)r * 3 * N + i];
        else mb_velocities(N, v, m, S.kT, S.seed, (uint32_t)r, (uint32_t)step0);
        cons_project_v(C, pairs, x, v);
        memset(f, 0, sizeof(double) * 3 * (size_t)N);
        orc_ff(&S, x, f, NULL);
        orc_stats st;
        stats_init(&st, C, n_blocks, n_steps - n_equil);
        for (int64_t t = 0; t < n_steps; ++t) {
            const uint32_t step = (uint32_t)(step0 + (uint64_t)t);
            for (int i = 0; i < 3 * N; ++i) v[i] += 0.5 * dt * f[i] / m;                  /* B */
            cons_project_v(C, pairs, x, v);
            memcpy(xo, x, sizeof(double) * 3 * (size_t)N);                                /* A */
            for (int i = 0; i < 3 * N; ++i) x[i] += 0.5 * dt * v[i];
            cons_shake(C, pairs, dr, xo, x, v, 0.5 * dt);
            cons_project_v(C, pairs, x, v);
            if (S.gamma > 0) {                                                            /* O */
                for (int i = 0; i < N; ++i) {
                    double xi[3];
                    orc_normals3(S.seed, (uint32_t)i, (uint32_t)r, step, 0u, xi);
                    for (int k = 0; k < 3; ++k) v[3 * i + k] = c1 * v[3 * i + k] + c2 * xi[k];
                }
                cons_project_v(C, pairs, x, v);
            }
            memcpy(xo, x, sizeof(double) * 3 * (size_t)N);                                /* A */
            for (int i = 0; i < 3 * N; ++i) x[i] += 0.5 * dt * v[i];
            cons_shake(C, pairs, dr, xo, x, v, 0.5 * dt);
            cons_project_v(C, pairs, x, v);
            memset(f, 0, sizeof(double) * 3 * (size_t)N);
            orc_ff(&S, x, f, NULL);
            for (int i = 0; i < 3 * N; ++i) v[i] += 0.5 * dt * f[i] / m;                  /* B */
            cons_project_v(C, pairs, x, v);
            if (t >= n_equil) {
                for (int j = 0; j < C; ++j) {
                    const int a = pairs[2 * j], b = pairs[2 * j + 1];
                    double fu = 0;
                    for (int k = 0; k < 3; ++k) fu += (f[3 * a + k] - f[3 * b + k]) * (x[3 * a + k] - x[3 * b + k]);
                    const double F = -0.5 * fu / dr[j] - 2.0 * S.kT / dr[j];
                    smp[j] = -F;              /* stats_finish returns -kappa mean: kappa = 1 */
                }
                stats_add(&st, t - n_equil, smp);
            }
        }
        stats_finish(&st, one, mf + (size_t)r * C, se + (size_t)r * C, sd + (size_t)r * C);
        stats_free(&st);
        if (x_out) memcpy(x_out + (size_t)r * 3 * N, x, sizeof(double) * 3 * (size_t)N);
        if (v_out) memcpy(v_out + (size_t)r * 3 * N, v, sizeof(double) * 3 * (size_t)N);
    }
    free(x); free(xo); free(v); free(f); free(smp); free(one);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* One-dimensional harmonic test systems that reuse the same integrator and */
/* label statistics: a particle in U(x) = a/2 (x - c)^2, optionally with a   */
/* restraint kappa/2 (x - s0)^2 on the (non-periodic) CV s = x.             */
/* Used to pin BAOAB (exact configurational variance for harmonic forces)    */
/* and the restrained mean force (closed form).                             */
/* moments = {<x>, <x^2>} over steps past n_equil.                          */
/* ------------------------------------------------------------------------ */
void orc_harmonic1d(double a, double c, double kappa, double s0, double m, double kT, double dt,
                    double gamma, uint64_t seed, int64_t n_steps, int64_t n_equil, int n_blocks,
                    double* mf, double* se, double* sd, double* moments)
{
    double x[3] = {c, 0, 0}, v[3] = {0, 0, 0}, f[3] = {0, 0, 0};
    orc_stats st;
    stats_init(&st, 1, n_blocks, n_steps - n_equil);
    double sx = 0, sxx = 0;
    f[0] = -a * (x[0] - c) - kappa * (x[0] - s0);
    for (int64_t t = 0; t < n_steps; ++t) {
        /* a single bead moving in one dimension: only xi_x of each draw is used */
        baoab_pre(1, 1, x, v, f, m, dt, gamma, kT, seed, 0u, (uint32_t)t);
        f[0] = -a * (x[0] - c) - kappa * (x[0] - s0);
        baoab_post(1, 1, v, f, m, dt);
        if (t >= n_equil) {
            double d = x[0] - s0;
            stats_add(&st, t - n_equil, &d);
            sx += x[0]; sxx += x[0] * x[0];
        }
    }
    double kap[1] = {kappa};
    stats_finish(&st, kap, mf, se, sd);
    stats_free(&st);
    moments[0] = sx / (double)(n_steps - n_equil);
    moments[1] = sxx / (double)(n_steps - n_equil);
}

/* Label statistics on a given sample sequence (for tests of the block rule). */
void orc_label_stats(int64_t K, int C, int B, const double* d /* [K][C] */, const double* kappa,
                     double* mf, double* se, double* sd)
{
    orc_stats st;
    stats_init(&st, C, B, K);
    for (int64_t k = 0; k < K; ++k) stats_add(&st, k, d + k * C);
    stats_finish(&st, kappa, mf, se, sd);
    stats_free(&st);
}
