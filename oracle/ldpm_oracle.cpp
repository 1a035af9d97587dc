/*
 * ldpm_oracle.cpp -- plain, slow FP64 reference of one LDPM explicit central-difference step, and
 * the exact derivative of the same computation with respect to per-facet material parameters.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark load this library.  It shares no code, header or table with the CUDA library; both
 * read the same raw specimen geometry and parameters.
 *
 * What it computes follows arXiv 2603.13190 (LDPM solver comparison):
 *   Sec. 2, Eq. (1)           facet strain e = P^T [[u]] / l from the rigid-body jump
 *   Sec. 2, Eq. (2a)-(2b)     particle force and moment balance, sum over facets of A P t
 *   Sec. 2, A = A0 n.n0       projected facet area
 *   Sec. 3, M q'' + f_int = f_ext with a lumped (diagonal) mass, central-difference integration
 *                             (the explicit solvers AE and JA, Sec. 3.2)
 *   Sec. 3.2.5                lumped mass: tetrahedron mass split equally over its 4 nodes,
 *                             isotropic rotary inertia m d^2 / 10
 *   App. A.1                  fracture law for e_N > 0
 *   App. A.2                  compressive law for e_N <= 0
 *   App. A.3                  frictional shear for e_N <= 0
 *   Sec. 4 (list of metrics)  energy balance 100 |W_ext - W_int - W_kin| / W_ext
 *
 * Readings where the paper is silent (each is also listed in the design notes):
 *   - central difference is written in its velocity form (half-step kick, drift, force, half-step
 *     kick); velocities are kept at whole steps;
 *   - the strain increment of a step is the difference of total strains (e_prev is stored);
 *   - t_old and e_old of the fracture law are the effective traction and effective strain of the
 *     previous step, recomputed from the stored traction and strain vectors;
 *   - e_max is updated only in the fracture branch; omega is evaluated at the current strain;
 *   - e_N > 0 selects the fracture branch, e_N <= 0 the compression/friction branch;
 *   - e_V of a tetrahedron is its linearised volumetric strain Delta V / (3 V0) = (1/3) div u;
 *   - in the fracture branch an effective strain below 1e-150 (where t/e is 0/0 in floating point)
 *     takes the elastic limit t = E e;
 *   - k_t > 0: on reloading from zero effective traction, only the part of the effective-strain
 *     increment above e_tr = k_t (e_max - sigma_bt / E0) counts (k_t = 0: the clamp alone);
 *   - r_s != 0 enters H_0 through H_s = r_s E0; the paper gives no law for the cohesion
 *     degradation it mentions, so sigma_s stays constant;
 *   - E_Nc = E_d when -t_N,old > sigma_c0, as written.
 *
 * Derivatives (the paper has none; they serve the adjoint of the explicit step).  The law and the
 * step are templates over the scalar type.  Instantiated with `double` they are the reference step;
 * instantiated with a forward-mode dual number they carry, next to every value, its derivative along
 * given directions of the per-facet parameters (E0, alpha, sigma_t), through every operation of the
 * same code.  Where an operation is not differentiable (sqrt at 0, a max or clamp at its switch
 * point, |x| at 0) the derivative of the branch the value takes is used, and sqrt'(0) is taken as 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <type_traits>
#include <vector>

#define ORC_PI 3.14159265358979323846
/* effective strains below this are treated as zero in the fracture law (squares would underflow) */
#define ORC_TINY_STRAIN 1e-150

/* ------------------------------------------------------------------------------------------ */
/* Forward-mode dual number: value v and its derivatives d[0..D) along D directions.             */
/* ------------------------------------------------------------------------------------------ */
template <int D>
struct Dual {
    double v;
    double d[D];
    Dual() : v(0.0) { for (int i = 0; i < D; ++i) d[i] = 0.0; }
    Dual(double x) : v(x) { for (int i = 0; i < D; ++i) d[i] = 0.0; }
};
template <int D> Dual<D> operator+(const Dual<D> &a, const Dual<D> &b) { Dual<D> r(a.v + b.v); for (int i = 0; i < D; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
template <int D> Dual<D> operator-(const Dual<D> &a, const Dual<D> &b) { Dual<D> r(a.v - b.v); for (int i = 0; i < D; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
template <int D> Dual<D> operator-(const Dual<D> &a) { Dual<D> r(-a.v); for (int i = 0; i < D; ++i) r.d[i] = -a.d[i]; return r; }
template <int D> Dual<D> operator*(const Dual<D> &a, const Dual<D> &b) { Dual<D> r(a.v * b.v); for (int i = 0; i < D; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
template <int D> Dual<D> operator/(const Dual<D> &a, const Dual<D> &b)
{
    Dual<D> r(a.v / b.v);
    for (int i = 0; i < D; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) / b.v; /* (a/b)' = (a' - (a/b) b') / b */
    return r;
}
template <int D> Dual<D> operator+(const Dual<D> &a, double b) { return a + Dual<D>(b); }
template <int D> Dual<D> operator+(double a, const Dual<D> &b) { return Dual<D>(a) + b; }
template <int D> Dual<D> operator-(const Dual<D> &a, double b) { return a - Dual<D>(b); }
template <int D> Dual<D> operator-(double a, const Dual<D> &b) { return Dual<D>(a) - b; }
template <int D> Dual<D> operator*(const Dual<D> &a, double b) { return a * Dual<D>(b); }
template <int D> Dual<D> operator*(double a, const Dual<D> &b) { return Dual<D>(a) * b; }
template <int D> Dual<D> operator/(const Dual<D> &a, double b) { return a / Dual<D>(b); }
template <int D> Dual<D> operator/(double a, const Dual<D> &b) { return Dual<D>(a) / b; }
template <int D> Dual<D> &operator+=(Dual<D> &a, const Dual<D> &b) { a = a + b; return a; }
template <int D> Dual<D> &operator-=(Dual<D> &a, const Dual<D> &b) { a = a - b; return a; }
template <int D> Dual<D> &operator*=(Dual<D> &a, const Dual<D> &b) { a = a * b; return a; }
template <int D> Dual<D> &operator/=(Dual<D> &a, const Dual<D> &b) { a = a / b; return a; }
/* comparisons act on the value */
template <int D> bool operator<(const Dual<D> &a, const Dual<D> &b) { return a.v < b.v; }
template <int D> bool operator>(const Dual<D> &a, const Dual<D> &b) { return a.v > b.v; }
template <int D> bool operator<=(const Dual<D> &a, const Dual<D> &b) { return a.v <= b.v; }
template <int D> bool operator<(const Dual<D> &a, double b) { return a.v < b; }
template <int D> bool operator>(const Dual<D> &a, double b) { return a.v > b; }
template <int D> bool operator<=(const Dual<D> &a, double b) { return a.v <= b; }
template <int D> Dual<D> sqrt(const Dual<D> &a)
{
    Dual<D> r(sqrt(a.v));
    for (int i = 0; i < D; ++i) r.d[i] = r.v > 0.0 ? a.d[i] / (2.0 * r.v) : 0.0;
    return r;
}
template <int D> Dual<D> exp(const Dual<D> &a)
{
    Dual<D> r(exp(a.v));
    for (int i = 0; i < D; ++i) r.d[i] = r.v * a.d[i];
    return r;
}
template <int D> Dual<D> sin(const Dual<D> &a)
{
    Dual<D> r(sin(a.v));
    const double c = cos(a.v);
    for (int i = 0; i < D; ++i) r.d[i] = c * a.d[i];
    return r;
}
template <int D> Dual<D> cos(const Dual<D> &a)
{
    Dual<D> r(cos(a.v));
    const double s = sin(a.v);
    for (int i = 0; i < D; ++i) r.d[i] = -s * a.d[i];
    return r;
}
/* d atan2(y, x) = (x dy - y dx) / (x^2 + y^2) */
template <int D> Dual<D> atan2(const Dual<D> &y, const Dual<D> &x)
{
    Dual<D> r(atan2(y.v, x.v));
    const double den = x.v * x.v + y.v * y.v;
    for (int i = 0; i < D; ++i) r.d[i] = den > 0.0 ? (x.v * y.d[i] - y.v * x.d[i]) / den : 0.0;
    return r;
}
template <int D> Dual<D> pow(const Dual<D> &a, double n)
{
    Dual<D> r(pow(a.v, n));
    const double g = n * pow(a.v, n - 1.0);
    for (int i = 0; i < D; ++i) r.d[i] = g * a.d[i];
    return r;
}
template <int D> Dual<D> fabs(const Dual<D> &a) { return a.v < 0.0 ? -a : a; }

static inline double value_of(double x) { return x; }
template <int D> static inline double value_of(const Dual<D> &x) { return x.v; }

typedef struct {
    double rho, E0, alpha, sigma_t, l_t, r_st, n_t, sigma_c0, Hc0_E0, Hc1_E0, kc0, kc1, kc2, kc3,
        mu0, mu_inf, sigma_N0, Ed_E0, beta, k_t, r_s;
    int32_t elastic; /* 1: linear elastic facets, t = E e (paper Sec. 4.1 benchmark) */
    int32_t pad_;
} orc_material;

typedef struct {
    int32_t N, T, F;
    orc_material mat;
    double dt, ramp_time;
    /* geometry */
    double *x;                      /* [N][3] */
    int32_t *tet;                   /* [T][4] */
    double *gradN;                  /* [T][4][3] */
    int32_t *fi, *fj, *ft;          /* [F] */
    double *n, *m, *lv, *ci, *cj;   /* [F][3] local frame, arms from I and J to the facet centroid */
    double *len, *area;             /* [F] */
    double *mass;                   /* [N][6] lumped mass per DOF */
    int32_t *bc_mask;               /* [N][6] */
    double *bc_vel, *f_ext;         /* [N][6] */
    /* state */
    int64_t step;
    double *q, *v;                  /* [N][6] */
    double *f_asm;                  /* [N][6] sum over facets of the force/moment acting on the node */
    double *t_loc;                  /* [F][3] tractions (t_N, t_M, t_L) */
    double *emax;                   /* [F] */
    double *e_prev;                 /* [F][3] strain of the current state */
    double *F_facet;                /* [F][3] facet force acting on I: A P t */
    double W_int, W_ext, W_kin0;
    /* per-facet E0, alpha, sigma_t ([F] each), or null: the material's values for every facet */
    double *pE0, *palpha, *psig;
} orc_model;

extern "C" {
void orc_facet_law(const orc_material *p, double l, const double e[3], const double de[3], double eV,
                   const double t_old[3], double emax_old, double t_new[3], double *emax_new);
void orc_facet_law_jacobian(const orc_material *p, double l, const double in[14], double out[4], double jac[56]);
void orc_destroy(orc_model *M);
orc_model *orc_create(int32_t N, int32_t T, int32_t F, const double *x, const double *diameter, const int32_t *tet,
                      const int32_t *fpi, const int32_t *fpj, const int32_t *ftet, const double *fvtx,
                      const double *mass_in, const double *inertia_in, const orc_material *mat, double dt,
                      const int32_t *bc_mask, const double *bc_vel, double ramp_time, const double *v0,
                      const double *f_ext);
int orc_step(orc_model *M, int64_t nsteps);
void orc_get_state(const orc_model *M, double *q, double *v, double *hist5, int64_t *step);
void orc_set_state(orc_model *M, const double *q, const double *v, const double *hist5, int64_t step);
void orc_energy(const orc_model *M, double out[4], double reaction[12]);
void orc_facet_forces(const orc_model *M, double *F3, double *f6);
void orc_strains(const orc_model *M, const double *q, double *e3, double *eV);
void orc_elastic_force(const orc_model *M, const double *q, double *f6);
double orc_lambda_max(const orc_model *M, const double *x0, int32_t iters);
void orc_geometry(const orc_model *M, double *n3, double *len, double *area, double *mass6, double *ci3,
                  double *cj3);
int32_t orc_sizes(const orc_model *M, int32_t *NTF);
void orc_facet_march(const orc_material *p, double l, int64_t n, const double *path, const double *eV,
                     double *t_out, double *emax_out);
void orc_metrics(const orc_model *M, double *w, double *eV);
void orc_set_bc(orc_model *M, const int32_t *mask, const double *vel, double ramp_time);
void orc_set_facet_params(orc_model *M, const double *E0, const double *alpha, const double *sigma_t);
void orc_perturb(orc_model *M, const double *dq);
int orc_tangent(const orc_model *M, int64_t nsteps, const double *seed, int32_t nd, const double *dE0,
                const double *dalpha, const double *dsigma_t, double *J, double *dJ);
}

static void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* ramp(t) = clamp(t / ramp_time, 0, 1); a prescribed DOF moves at bc_vel * ramp(t). */
static double ramp(const orc_model *M, double t)
{
    if (M->ramp_time <= 0.0) return 1.0;
    double r = t / M->ramp_time;
    if (r < 0.0) r = 0.0;
    if (r > 1.0) r = 1.0;
    return r;
}

/* ------------------------------------------------------------------------------------------ */
/* Constitutive law, App. A.  Inputs: strain e (local N, M, L), its increment over the step de,  */
/* the tetrahedron's volumetric strain eV, the facet length l, the previous tractions t_old and */
/* maximum effective strain.  Outputs the new tractions and e_max.                              */
/* ------------------------------------------------------------------------------------------ */
template <class S>
static void facet_law(const orc_material *p, S E0, S alpha, S sigma_t, double l, const S e[3], const S de[3],
                      S eV, const S t_old[3], S emax_old, S t_new[3], S *emax_new)
{
    *emax_new = emax_old;
    if (p->elastic) {
        /* Sec. 2: t = E e with E = E0 diag(1, alpha, alpha). */
        t_new[0] = E0 * e[0];
        t_new[1] = alpha * E0 * e[1];
        t_new[2] = alpha * E0 * e[2];
        return;
    }
    if (e[0] > 0.0) {
        /* App. A.1, fracture.  Effective strain e = sqrt(e_N^2 + alpha (e_M^2 + e_L^2)). */
        S eT2 = e[1] * e[1] + e[2] * e[2];
        S eeff = sqrt(e[0] * e[0] + alpha * eT2);
        if (eeff < ORC_TINY_STRAIN) {
            /* The ratio t / e of the expressions below is 0/0 at e = 0; its limit on the elastic
             * path is E0, so a vanishing effective strain responds elastically, t = E e. */
            t_new[0] = E0 * e[0];
            t_new[1] = alpha * E0 * e[1];
            t_new[2] = alpha * E0 * e[2];
            *emax_new = emax_old > eeff ? emax_old : eeff;
            return;
        }
        /* Coupling angle, tan(omega) = e_N / sqrt(alpha (e_M^2 + e_L^2)). */
        S omega = atan2(e[0], sqrt(alpha * eT2));
        S s = sin(omega), c = cos(omega);
        double r2 = p->r_st * p->r_st;
        /* sigma_0(omega) = sigma_t (-s + sqrt(s^2 + 4 alpha c^2 / r^2)) / (2 alpha c^2 / r^2).
         * Multiplying numerator and denominator by (s + sqrt(s^2 + 4 alpha c^2 / r^2)) gives the
         * same value as 2 sigma_t / (s + sqrt(s^2 + 4 alpha c^2 / r^2)), which stays finite at
         * omega = pi/2 (c = 0); that form is used. */
        S sigma0 = 2.0 * sigma_t / (s + sqrt(s * s + 4.0 * alpha * c * c / r2));
        /* H_0(omega) = H_s/alpha + (H_t - H_s/alpha) (2 omega / pi)^n_t,
         * H_t = 2 E0 / (l_t / l - 1), H_s = r_s E0. */
        S Ht = 2.0 * E0 / (p->l_t / l - 1.0);
        S Hs = p->r_s * E0;
        S H0 = Hs / alpha + (Ht - Hs / alpha) * pow(2.0 * omega / ORC_PI, p->n_t);
        S e0 = sigma0 / E0;
        S emax = emax_old > eeff ? emax_old : eeff;
        S over = emax - e0 > 0.0 ? emax - e0 : 0.0;
        S sigma_bt = sigma0 * exp(-H0 * over / sigma0);
        /* Incrementally elastic effective traction: t = t_old + E0 (e - e_old), then the vertical
         * return onto 0 <= t <= sigma_bt. */
        S e_prev[3] = {e[0] - de[0], e[1] - de[1], e[2] - de[2]};
        S e_old = sqrt(e_prev[0] * e_prev[0] + alpha * (e_prev[1] * e_prev[1] + e_prev[2] * e_prev[2]));
        S t_eff_old = sqrt(t_old[0] * t_old[0] + (t_old[1] * t_old[1] + t_old[2] * t_old[2]) / alpha);
        S de_eff = eeff - e_old;
        if (p->k_t > 0.0 && t_eff_old <= 0.0 && de_eff > 0.0) {
            /* Reloading from zero traction: the traction stays zero until the effective strain
             * reaches e_tr = k_t (e_max - sigma_bt / E0), then grows elastically (App. A.1).  With
             * k_t = 0, e_tr = 0 and the whole increment counts (the clamp alone). */
            S e_tr = p->k_t * (emax - sigma_bt / E0);
            if (e_tr > e_old) de_eff = eeff > e_tr ? eeff - e_tr : S(0.0);
        }
        S t = t_eff_old + E0 * de_eff;
        if (t < 0.0) t = 0.0;
        if (t > sigma_bt) t = sigma_bt;
        /* t_N = (t/e) e_N, t_M = alpha (t/e) e_M, t_L = alpha (t/e) e_L */
        t_new[0] = t / eeff * e[0];
        t_new[1] = alpha * t / eeff * e[1];
        t_new[2] = alpha * t / eeff * e[2];
        *emax_new = emax;
        return;
    }
    /* App. A.2, compression: t_N incrementally elastic with E_Nc, within -sigma_bc <= t_N <= 0. */
    S Ed = p->Ed_E0 * E0;
    S ENc = (-t_old[0] <= p->sigma_c0) ? E0 : Ed;
    S tN = t_old[0] + ENc * de[0];
    S eD = e[0] - eV;
    S eDV = eV + p->beta * eD;
    S ec0 = p->sigma_c0 / E0;
    S ec1 = p->kc0 * ec0;
    S eV0 = p->kc3 * p->sigma_c0 / E0;
    S rDV = (eV <= 0.0) ? -fabs(eD) / (eV - eV0) : fabs(eD) / eV0;
    S Hc0 = p->Hc0_E0 * E0, Hc1 = p->Hc1_E0 * E0;
    S mac = rDV - p->kc1 > 0.0 ? rDV - p->kc1 : 0.0;
    S Hc = (Hc0 - Hc1) / (1.0 + p->kc2 * mac) + Hc1;
    S sigma_c1 = p->sigma_c0 + (ec1 - ec0) * Hc;
    S sigma_bc;
    if (-eDV <= 0.0) {
        sigma_bc = p->sigma_c0;
    } else if (-eDV <= ec1) {
        S o = -eDV - ec0 > 0.0 ? -eDV - ec0 : 0.0;
        sigma_bc = p->sigma_c0 + o * Hc;
    } else {
        sigma_bc = sigma_c1 * exp((-eDV - ec1) * Hc / sigma_c1);
    }
    if (tN < -sigma_bc) tN = -sigma_bc;
    if (tN > 0.0) tN = 0.0;
    /* App. A.3, friction: elastic shear trial with stiffness alpha E0, yield surface
     * phi = sqrt(t_M^2 + t_L^2) - sigma_bs(t_N), associated flow.  With the shear stiffness the
     * same in M and L, the return along the normal is a radial scaling onto the circle. */
    S tM = t_old[1] + alpha * E0 * de[1];
    S tL = t_old[2] + alpha * E0 * de[2];
    S sigma_s = p->r_st * sigma_t;
    double dmu = p->mu0 - p->mu_inf;
    S sigma_bs = sigma_s + dmu * p->sigma_N0 - p->mu_inf * tN - dmu * p->sigma_N0 * exp(tN / p->sigma_N0);
    S tau = sqrt(tM * tM + tL * tL);
    if (tau > sigma_bs) {
        tM *= sigma_bs / tau;
        tL *= sigma_bs / tau;
    }
    t_new[0] = tN;
    t_new[1] = tM;
    t_new[2] = tL;
}

void orc_facet_law(const orc_material *p, double l, const double e[3], const double de[3], double eV,
                   const double t_old[3], double emax_old, double t_new[3], double *emax_new)
{
    facet_law<double>(p, p->E0, p->alpha, p->sigma_t, l, e, de, eV, t_old, emax_old, t_new, emax_new);
}

/* ------------------------------------------------------------------------------------------ */
/* Kinematics, Sec. 2, Eq. (1).                                                                 */
/* ------------------------------------------------------------------------------------------ */
template <class S>
static void facet_strain(const orc_model *M, const S *q, int32_t k, S e[3])
{
    const S *uI = q + 6 * (size_t)M->fi[k], *uJ = q + 6 * (size_t)M->fj[k];
    const double *cI = M->ci + 3 * (size_t)k, *cJ = M->cj + 3 * (size_t)k;
    S jump[3];
    for (int a = 0; a < 3; ++a) {
        const int b = (a + 1) % 3, c = (a + 2) % 3;
        const S rI = uI[3 + b] * cI[c] - uI[3 + c] * cI[b]; /* (theta_I x c_I)_a */
        const S rJ = uJ[3 + b] * cJ[c] - uJ[3 + c] * cJ[b]; /* (theta_J x c_J)_a */
        jump[a] = uJ[a] + rJ - uI[a] - rI;
    }
    double l = M->len[k];
    const double *n = M->n + 3 * (size_t)k, *m = M->m + 3 * (size_t)k, *lv = M->lv + 3 * (size_t)k;
    e[0] = (n[0] * jump[0] + n[1] * jump[1] + n[2] * jump[2]) / l;
    e[1] = (m[0] * jump[0] + m[1] * jump[1] + m[2] * jump[2]) / l;
    e[2] = (lv[0] * jump[0] + lv[1] * jump[1] + lv[2] * jump[2]) / l;
}

/* Linearised volumetric strain of tetrahedron t: (1/3) sum_i gradN_i . u_i  (App. A.2 e_V). */
template <class S>
static S tet_volumetric_strain(const orc_model *M, const S *q, int32_t t)
{
    S dv = 0.0;
    for (int i = 0; i < 4; ++i) {
        const double *g = M->gradN + 12 * (size_t)t + 3 * i;
        const S *u = q + 6 * (size_t)M->tet[4 * (size_t)t + i];
        dv += g[0] * u[0] + g[1] * u[1] + g[2] * u[2];
    }
    return dv / 3.0;
}

/* F_k = A_k P_k t_k; node I receives +F_k and moment c_I x F_k, node J the opposite force and
 * moment -c_J x F_k (Eq. (2a)-(2b) summed over each node's facets). */
template <class S>
static void facet_force(const orc_model *M, int32_t k, const S t[3], S F[3])
{
    for (int a = 0; a < 3; ++a)
        F[a] = M->area[k] * (M->n[3 * k + a] * t[0] + M->m[3 * k + a] * t[1] + M->lv[3 * k + a] * t[2]);
}

template <class S>
static void assemble(const orc_model *M, const S *F, S *f_asm)
{
    for (size_t i = 0; i < 6 * (size_t)M->N; ++i) f_asm[i] = 0.0;
    for (int32_t k = 0; k < M->F; ++k) {
        const S *Fk = F + 3 * (size_t)k;
        const double *cI = M->ci + 3 * (size_t)k, *cJ = M->cj + 3 * (size_t)k;
        S *fI = f_asm + 6 * (size_t)M->fi[k], *fJ = f_asm + 6 * (size_t)M->fj[k];
        for (int a = 0; a < 3; ++a) {
            const int b = (a + 1) % 3, c = (a + 2) % 3;
            const S mI = cI[b] * Fk[c] - cI[c] * Fk[b]; /* (c_I x F)_a */
            const S mJ = cJ[b] * Fk[c] - cJ[c] * Fk[b]; /* (c_J x F)_a */
            fI[a] += Fk[a];
            fI[3 + a] += mI;
            fJ[a] -= Fk[a];
            fJ[3 + a] -= mJ;
        }
    }
}

/* Facet forces from the stored tractions, then the node sums. */
static void forces_from_history(orc_model *M)
{
    for (int32_t k = 0; k < M->F; ++k) facet_force(M, k, M->t_loc + 3 * (size_t)k, M->F_facet + 3 * (size_t)k);
    assemble(M, M->F_facet, M->f_asm);
}

/* ------------------------------------------------------------------------------------------ */
/* Set-up from raw geometry.                                                                    */
/* ------------------------------------------------------------------------------------------ */
void orc_destroy(orc_model *M)
{
    if (!M) return;
    void *ptrs[] = {M->x, M->tet, M->gradN, M->fi, M->fj, M->ft, M->n, M->m, M->lv, M->ci, M->cj, M->len,
                    M->area, M->mass, M->bc_mask, M->bc_vel, M->f_ext, M->q, M->v, M->f_asm, M->t_loc,
                    M->emax, M->e_prev, M->F_facet, M->pE0, M->palpha, M->psig};
    for (size_t i = 0; i < sizeof(ptrs) / sizeof(ptrs[0]); ++i) free(ptrs[i]);
    free(M);
}

/* Returns NULL on bad input.  mass_in / inertia_in may be NULL (then the Sec. 3.2.5 rule is used).
 * bc_mask / bc_vel / v0 / f_ext may be NULL (free, zero). */
orc_model *orc_create(int32_t N, int32_t T, int32_t F, const double *x, const double *diameter, const int32_t *tet,
                      const int32_t *fpi, const int32_t *fpj, const int32_t *ftet, const double *fvtx,
                      const double *mass_in, const double *inertia_in, const orc_material *mat, double dt,
                      const int32_t *bc_mask, const double *bc_vel, double ramp_time, const double *v0,
                      const double *f_ext)
{
    if (N <= 0 || T < 0 || F <= 0 || !x || !fpi || !fpj || !fvtx || !mat) return NULL;
    orc_model *M = (orc_model *)calloc(1, sizeof(orc_model));
    M->N = N;
    M->T = T;
    M->F = F;
    M->mat = *mat;
    M->dt = dt;
    M->ramp_time = ramp_time;
    size_t n6 = 6 * (size_t)N;
    M->x = (double *)malloc(sizeof(double) * 3 * N);
    memcpy(M->x, x, sizeof(double) * 3 * N);
    M->tet = (int32_t *)calloc(4 * (size_t)T + 1, sizeof(int32_t));
    if (T) memcpy(M->tet, tet, sizeof(int32_t) * 4 * T);
    M->gradN = (double *)calloc(12 * (size_t)T + 1, sizeof(double));
    M->fi = (int32_t *)malloc(sizeof(int32_t) * F);
    M->fj = (int32_t *)malloc(sizeof(int32_t) * F);
    M->ft = (int32_t *)malloc(sizeof(int32_t) * F);
    M->n = (double *)malloc(sizeof(double) * 3 * F);
    M->m = (double *)malloc(sizeof(double) * 3 * F);
    M->lv = (double *)malloc(sizeof(double) * 3 * F);
    M->ci = (double *)malloc(sizeof(double) * 3 * F);
    M->cj = (double *)malloc(sizeof(double) * 3 * F);
    M->len = (double *)malloc(sizeof(double) * F);
    M->area = (double *)malloc(sizeof(double) * F);
    M->mass = (double *)calloc(n6, sizeof(double));
    M->bc_mask = (int32_t *)calloc(n6, sizeof(int32_t));
    M->bc_vel = (double *)calloc(n6, sizeof(double));
    M->f_ext = (double *)calloc(n6, sizeof(double));
    M->q = (double *)calloc(n6, sizeof(double));
    M->v = (double *)calloc(n6, sizeof(double));
    M->f_asm = (double *)calloc(n6, sizeof(double));
    M->t_loc = (double *)calloc(3 * (size_t)F, sizeof(double));
    M->emax = (double *)calloc(F, sizeof(double));
    M->e_prev = (double *)calloc(3 * (size_t)F, sizeof(double));
    M->F_facet = (double *)calloc(3 * (size_t)F, sizeof(double));
    if (bc_mask) memcpy(M->bc_mask, bc_mask, sizeof(int32_t) * n6);
    if (bc_vel) memcpy(M->bc_vel, bc_vel, sizeof(double) * n6);
    if (f_ext) memcpy(M->f_ext, f_ext, sizeof(double) * n6);

    /* Tetrahedra: shape-function gradients of the linear tetrahedron and the lumped mass.
     * With D = [x1-x0, x2-x0, x3-x0] (columns), grad N_1..3 are the rows of D^-1 and
     * grad N_0 = -(grad N_1 + grad N_2 + grad N_3). */
    double *node_mass = (double *)calloc(N, sizeof(double));
    for (int32_t t = 0; t < T; ++t) {
        const int32_t *v = M->tet + 4 * (size_t)t;
        double d1[3], d2[3], d3[3];
        for (int a = 0; a < 3; ++a) {
            d1[a] = x[3 * v[1] + a] - x[3 * v[0] + a];
            d2[a] = x[3 * v[2] + a] - x[3 * v[0] + a];
            d3[a] = x[3 * v[3] + a] - x[3 * v[0] + a];
        }
        double c23[3], c31[3], c12[3];
        cross3(d2, d3, c23);
        cross3(d3, d1, c31);
        cross3(d1, d2, c12);
        double det = dot3(d1, c23); /* 6 V (signed) */
        if (det == 0.0) {
            free(node_mass);
            orc_destroy(M);
            return NULL;
        }
        double *g = M->gradN + 12 * (size_t)t;
        for (int a = 0; a < 3; ++a) {
            g[3 + a] = c23[a] / det;
            g[6 + a] = c31[a] / det;
            g[9 + a] = c12[a] / det;
            g[a] = -(g[3 + a] + g[6 + a] + g[9 + a]);
        }
        double vol = fabs(det) / 6.0;
        for (int i = 0; i < 4; ++i) node_mass[v[i]] += mat->rho * vol / 4.0; /* Sec. 3.2.5 */
    }
    double dpos_min = INFINITY;
    for (int32_t i = 0; i < N; ++i)
        if (diameter && diameter[i] > 0.0 && diameter[i] < dpos_min) dpos_min = diameter[i];
    for (int32_t i = 0; i < N; ++i) {
        double mi = mass_in ? mass_in[i] : node_mass[i];
        double d = (diameter && diameter[i] > 0.0) ? diameter[i] : dpos_min;
        for (int a = 0; a < 3; ++a) {
            M->mass[6 * i + a] = mi;
            /* I_m = m d^2 / 10 (solid sphere), nodes with d = 0 use the smallest positive d */
            M->mass[6 * i + 3 + a] = inertia_in ? inertia_in[3 * i + a] : mi * d * d / 10.0;
        }
    }
    free(node_mass);

    /* Facets: n along IJ, a tangent pair (m, l), arms to the facet centroid, projected area. */
    for (int32_t k = 0; k < F; ++k) {
        int32_t I = fpi[k], J = fpj[k];
        if (I < 0 || I >= N || J < 0 || J >= N || I == J) {
            orc_destroy(M);
            return NULL;
        }
        M->fi[k] = I;
        M->fj[k] = J;
        M->ft[k] = ftet ? ftet[k] : -1;
        double d[3], nn[3];
        for (int a = 0; a < 3; ++a) d[a] = x[3 * J + a] - x[3 * I + a];
        double l = sqrt(dot3(d, d));
        for (int a = 0; a < 3; ++a) nn[a] = d[a] / l;
        /* Tangent m: the world axis least aligned with n, made orthogonal to n and normalised;
         * l = n x m.  (Any orthonormal tangent pair is allowed, Sec. 2.) */
        int ax = 0;
        for (int a = 1; a < 3; ++a)
            if (fabs(nn[a]) < fabs(nn[ax])) ax = a;
        double mm[3] = {0.0, 0.0, 0.0};
        mm[ax] = 1.0;
        double pr = dot3(mm, nn);
        for (int a = 0; a < 3; ++a) mm[a] -= pr * nn[a];
        double mn = sqrt(dot3(mm, mm));
        for (int a = 0; a < 3; ++a) mm[a] /= mn;
        double ll[3];
        cross3(nn, mm, ll);
        const double *p0 = fvtx + 9 * (size_t)k, *p1 = p0 + 3, *p2 = p0 + 6;
        double e1[3], e2[3], nc[3], xc[3];
        for (int a = 0; a < 3; ++a) {
            e1[a] = p1[a] - p0[a];
            e2[a] = p2[a] - p0[a];
            xc[a] = (p0[a] + p1[a] + p2[a]) / 3.0;
        }
        cross3(e1, e2, nc);
        double twoA0 = sqrt(dot3(nc, nc));
        if (!(l > 0.0) || !(twoA0 > 0.0)) {
            orc_destroy(M);
            return NULL;
        }
        /* A = A0 n . n0 (projected area; the facet orientation sign is irrelevant) */
        double A = 0.5 * twoA0 * fabs(dot3(nn, nc) / twoA0);
        for (int a = 0; a < 3; ++a) {
            M->n[3 * k + a] = nn[a];
            M->m[3 * k + a] = mm[a];
            M->lv[3 * k + a] = ll[a];
            M->ci[3 * k + a] = xc[a] - x[3 * I + a];
            M->cj[3 * k + a] = xc[a] - x[3 * J + a];
        }
        M->len[k] = l;
        M->area[k] = A;
    }

    /* Initial state: q = 0, zero history; prescribed DOFs start at their prescribed velocity. */
    for (size_t i = 0; i < n6; ++i) {
        M->v[i] = v0 ? v0[i] : 0.0;
        if (M->bc_mask[i] == 1) M->v[i] = 0.0;
        if (M->bc_mask[i] == 2) M->v[i] = M->bc_vel[i] * ramp(M, 0.0);
    }
    M->W_kin0 = 0.0;
    for (size_t i = 0; i < n6; ++i) M->W_kin0 += 0.5 * M->mass[i] * M->v[i] * M->v[i];
    return M;
}

/* ------------------------------------------------------------------------------------------ */
/* Time stepping.                                                                               */
/* ------------------------------------------------------------------------------------------ */

/* Total generalised force acting on each DOF, g = f_ext + R + f_asm, where R is the reaction on a
 * constrained DOF (zero on free DOFs).  On constrained DOFs g = mass * a with a the acceleration the
 * constraint imposes: 0 when fixed, (vbar(t + dt/2) - vbar(t - dt/2)) / dt when prescribed.  Returns
 * f_ext + R (the part the external world applies). */
template <class S>
static S ext_force_on_dof(const orc_model *M, size_t i, double t, const S *f_asm)
{
    if (M->bc_mask[i] == 0) return S(M->f_ext[i]);
    double a = 0.0;
    if (M->bc_mask[i] == 2) a = M->bc_vel[i] * (ramp(M, t + 0.5 * M->dt) - ramp(M, t - 0.5 * M->dt)) / M->dt;
    return M->mass[i] * a - f_asm[i];
}

/* The evolving part of a trajectory in scalar type S, and the per-facet parameters it runs with
 * (null: the material's value for every facet). */
template <class S>
struct Traj {
    S *q, *v, *f_asm, *t_loc, *emax, *e_prev, *F;
    const S *E0, *alpha, *sigma_t;
};

/* One facet pass at the current q: strains, constitutive update, facet forces, node sums. */
template <class S>
static void facet_pass(const orc_model *M, Traj<S> &T)
{
    std::vector<S> eV((size_t)M->T + 1);
    for (int32_t t = 0; t < M->T; ++t) eV[t] = tet_volumetric_strain(M, T.q, t);
    for (int32_t k = 0; k < M->F; ++k) {
        S e[3], de[3], tn[3], em;
        facet_strain(M, T.q, k, e);
        for (int a = 0; a < 3; ++a) de[a] = e[a] - T.e_prev[3 * k + a];
        S ev = M->ft[k] >= 0 ? eV[M->ft[k]] : e[0];
        const S E0 = T.E0 ? T.E0[k] : S(M->mat.E0);
        const S alpha = T.alpha ? T.alpha[k] : S(M->mat.alpha);
        const S sigma_t = T.sigma_t ? T.sigma_t[k] : S(M->mat.sigma_t);
        facet_law<S>(&M->mat, E0, alpha, sigma_t, M->len[k], e, de, ev, T.t_loc + 3 * (size_t)k, T.emax[k], tn, &em);
        for (int a = 0; a < 3; ++a) {
            T.t_loc[3 * k + a] = tn[a];
            T.e_prev[3 * k + a] = e[a];
        }
        T.emax[k] = em;
        facet_force(M, k, tn, T.F + 3 * (size_t)k);
    }
    assemble(M, T.F, T.f_asm);
}

/* `nsteps` central-difference steps of trajectory T from step counter *step.  With S = double the
 * energies are accumulated into W[0] = W_int, W[1] = W_ext (W not null).  With `seed` given, after every step
 * J += sum over constrained DOFs i of seed_i (f_ext + R)_i. */
template <class S>
static void run_steps(const orc_model *M, Traj<S> &T, int64_t nsteps, int64_t *step, double *W, const double *seed,
                      S *J)
{
    size_t n6 = 6 * (size_t)M->N;
    double dt = M->dt;
    std::vector<S> dq(n6), vh(n6), g_old(n6), fint_old(n6);
    for (int64_t s = 0; s < nsteps; ++s) {
        double t = (double)*step * dt;
        /* half kick and drift: v_{n+1/2} = v_n + dt/2 a_n ; q_{n+1} = q_n + dt v_{n+1/2} */
        for (size_t i = 0; i < n6; ++i) {
            g_old[i] = ext_force_on_dof(M, i, t, T.f_asm);
            fint_old[i] = -T.f_asm[i];
            if (M->bc_mask[i] == 0)
                vh[i] = T.v[i] + 0.5 * dt * (M->f_ext[i] + T.f_asm[i]) / M->mass[i];
            else if (M->bc_mask[i] == 1)
                vh[i] = 0.0;
            else
                vh[i] = M->bc_vel[i] * ramp(M, t + 0.5 * dt);
            dq[i] = dt * vh[i];
            T.q[i] += dq[i];
        }
        /* internal forces at q_{n+1} */
        facet_pass(M, T);
        *step += 1;
        double t1 = (double)*step * dt;
        /* energies (trapezoid rule on each DOF's increment) and the second half kick */
        for (size_t i = 0; i < n6; ++i) {
            S g_new = ext_force_on_dof(M, i, t1, T.f_asm);
            if constexpr (std::is_same<S, double>::value) {
                if (W) {
                    W[1] += 0.5 * (g_old[i] + g_new) * dq[i];
                    W[0] += 0.5 * (fint_old[i] - T.f_asm[i]) * dq[i];
                }
            }
            if (seed && M->bc_mask[i] != 0) *J += seed[i] * g_new;
            if (M->bc_mask[i] == 0)
                T.v[i] = vh[i] + 0.5 * dt * (M->f_ext[i] + T.f_asm[i]) / M->mass[i];
            else if (M->bc_mask[i] == 1)
                T.v[i] = 0.0;
            else
                T.v[i] = M->bc_vel[i] * ramp(M, t1);
        }
    }
}

int orc_step(orc_model *M, int64_t nsteps)
{
    Traj<double> T{M->q, M->v, M->f_asm, M->t_loc, M->emax, M->e_prev, M->F_facet, M->pE0, M->palpha, M->psig};
    double W[2] = {M->W_int, M->W_ext};
    run_steps<double>(M, T, nsteps, &M->step, W, NULL, NULL);
    M->W_int = W[0];
    M->W_ext = W[1];
    size_t n6 = 6 * (size_t)M->N;
    for (size_t i = 0; i < n6; ++i)
        if (!isfinite(M->q[i]) || !isfinite(M->v[i])) return -5;
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* State exchange.  History per facet: t_N, the tangential traction as a global vector          */
/* t_M m + t_L l (3 values), e_max.                                                             */
/* ------------------------------------------------------------------------------------------ */
void orc_get_state(const orc_model *M, double *q, double *v, double *hist5, int64_t *step)
{
    size_t n6 = 6 * (size_t)M->N;
    if (q) memcpy(q, M->q, sizeof(double) * n6);
    if (v) memcpy(v, M->v, sizeof(double) * n6);
    if (hist5)
        for (int32_t k = 0; k < M->F; ++k) {
            const double *t = M->t_loc + 3 * (size_t)k;
            hist5[5 * k] = t[0];
            for (int a = 0; a < 3; ++a) hist5[5 * k + 1 + a] = t[1] * M->m[3 * k + a] + t[2] * M->lv[3 * k + a];
            hist5[5 * k + 4] = M->emax[k];
        }
    if (step) *step = M->step;
}

void orc_set_state(orc_model *M, const double *q, const double *v, const double *hist5, int64_t step)
{
    size_t n6 = 6 * (size_t)M->N;
    memcpy(M->q, q, sizeof(double) * n6);
    memcpy(M->v, v, sizeof(double) * n6);
    for (int32_t k = 0; k < M->F; ++k) {
        const double *h = hist5 + 5 * (size_t)k;
        M->t_loc[3 * k] = h[0];
        M->t_loc[3 * k + 1] = dot3(h + 1, M->m + 3 * (size_t)k);
        M->t_loc[3 * k + 2] = dot3(h + 1, M->lv + 3 * (size_t)k);
        M->emax[k] = h[4];
        facet_strain(M, M->q, k, M->e_prev + 3 * (size_t)k);
    }
    M->step = step;
    forces_from_history(M);
    M->W_int = M->W_ext = 0.0;
    M->W_kin0 = 0.0;
    for (size_t i = 0; i < n6; ++i) M->W_kin0 += 0.5 * M->mass[i] * M->v[i] * M->v[i];
}

/* out = {W_ext, W_int, W_kin, error %}; reaction = sums of f_ext + R over fixed DOFs (6 values,
 * one per DOF component) then over prescribed DOFs (6 values).  Error % (Sec. 4):
 * 100 |W_ext + W_kin0 - W_int - W_kin| / (|W_ext| + W_kin0), the initial kinetic energy counted
 * as supplied energy (it is zero in the loaded benchmarks, where this is the paper's formula). */
void orc_energy(const orc_model *M, double out[4], double reaction[12])
{
    double Wk = 0.0;
    size_t n6 = 6 * (size_t)M->N;
    for (size_t i = 0; i < n6; ++i) Wk += 0.5 * M->mass[i] * M->v[i] * M->v[i];
    out[0] = M->W_ext;
    out[1] = M->W_int;
    out[2] = Wk;
    double den = fabs(M->W_ext) + M->W_kin0;
    out[3] = den > 0.0 ? 100.0 * fabs(M->W_ext + M->W_kin0 - M->W_int - Wk) / den : 0.0;
    if (reaction) {
        double t = (double)M->step * M->dt;
        for (int c = 0; c < 12; ++c) reaction[c] = 0.0;
        for (size_t i = 0; i < n6; ++i) {
            int mk = M->bc_mask[i];
            if (mk == 0) continue;
            reaction[(mk == 1 ? 0 : 6) + (int)(i % 6)] += ext_force_on_dof(M, i, t, M->f_asm);
        }
    }
}

/* Facet forces on I (global, [F][3]) and node sums ([N][6]) of the current state. */
void orc_facet_forces(const orc_model *M, double *F3, double *f6)
{
    if (F3) memcpy(F3, M->F_facet, sizeof(double) * 3 * (size_t)M->F);
    if (f6) memcpy(f6, M->f_asm, sizeof(double) * 6 * (size_t)M->N);
}

/* Strains at displacement q (local e per facet, [F][3]) and e_V per tetrahedron ([T]). */
void orc_strains(const orc_model *M, const double *q, double *e3, double *eV)
{
    if (e3)
        for (int32_t k = 0; k < M->F; ++k) facet_strain(M, q, k, e3 + 3 * (size_t)k);
    if (eV)
        for (int32_t t = 0; t < M->T; ++t) eV[t] = tet_volumetric_strain(M, q, t);
}

/* Node sums of the linear-elastic facet forces at displacement q (zero history): -K q. */
void orc_elastic_force(const orc_model *M, const double *q, double *f6)
{
    double *F = (double *)malloc(sizeof(double) * 3 * (size_t)M->F);
    for (int32_t k = 0; k < M->F; ++k) {
        double e[3], t[3];
        facet_strain(M, q, k, e);
        t[0] = M->mat.E0 * e[0];
        t[1] = M->mat.alpha * M->mat.E0 * e[1];
        t[2] = M->mat.alpha * M->mat.E0 * e[2];
        facet_force(M, k, t, F + 3 * (size_t)k);
    }
    assemble(M, F, f6);
    free(F);
}

/* Largest eigenvalue of M^-1 K (power iteration from x0, `iters` products).  The stable central-
 * difference step is 2 / sqrt(lambda_max) (the paper runs at about 90 % of it, Sec. 4.1). */
double orc_lambda_max(const orc_model *M, const double *x0, int32_t iters)
{
    size_t n6 = 6 * (size_t)M->N;
    double *x = (double *)malloc(sizeof(double) * n6);
    double *f = (double *)malloc(sizeof(double) * n6);
    memcpy(x, x0, sizeof(double) * n6);
    double lam = 0.0;
    for (int32_t it = 0; it < iters; ++it) {
        double nrm = 0.0;
        for (size_t i = 0; i < n6; ++i) nrm += M->mass[i] * x[i] * x[i];
        nrm = sqrt(nrm);
        for (size_t i = 0; i < n6; ++i) x[i] /= nrm;
        orc_elastic_force(M, x, f); /* f = -K x */
        double xKx = 0.0;
        for (size_t i = 0; i < n6; ++i) xKx -= x[i] * f[i];
        lam = xKx; /* x^T M x = 1 */
        for (size_t i = 0; i < n6; ++i) x[i] = -f[i] / M->mass[i];
    }
    free(x);
    free(f);
    return lam;
}

/* Read-only views used by tests. */
void orc_geometry(const orc_model *M, double *n3, double *len, double *area, double *mass6, double *ci3,
                  double *cj3)
{
    if (n3) memcpy(n3, M->n, sizeof(double) * 3 * (size_t)M->F);
    if (len) memcpy(len, M->len, sizeof(double) * M->F);
    if (area) memcpy(area, M->area, sizeof(double) * M->F);
    if (mass6) memcpy(mass6, M->mass, sizeof(double) * 6 * (size_t)M->N);
    if (ci3) memcpy(ci3, M->ci, sizeof(double) * 3 * (size_t)M->F);
    if (cj3) memcpy(cj3, M->cj, sizeof(double) * 3 * (size_t)M->F);
}

int32_t orc_sizes(const orc_model *M, int32_t *NTF) { NTF[0] = M->N; NTF[1] = M->T; NTF[2] = M->F; return 0; }

/* Drive one facet along a strain path: row i of `path` is the total strain after step i (the
 * increment is the difference to the previous row, the first measured from zero strain), eV[i] the
 * volumetric strain of its tetrahedron.  Writes the tractions and e_max after each step. */
void orc_facet_march(const orc_material *p, double l, int64_t n, const double *path, const double *eV,
                     double *t_out, double *emax_out)
{
    double t[3] = {0.0, 0.0, 0.0}, em = 0.0, e_prev[3] = {0.0, 0.0, 0.0};
    for (int64_t i = 0; i < n; ++i) {
        const double *e = path + 3 * i;
        double de[3] = {e[0] - e_prev[0], e[1] - e_prev[1], e[2] - e_prev[2]};
        double tn[3], emn;
        orc_facet_law(p, l, e, de, eV[i], t, em, tn, &emn);
        for (int a = 0; a < 3; ++a) {
            t[a] = tn[a];
            e_prev[a] = e[a];
            t_out[3 * i + a] = tn[a];
        }
        em = emn;
        emax_out[i] = em;
    }
}

/* Crack opening per facet (Sec. 4: w = sqrt(w_N^2 + w_M^2 + w_L^2), only positive inelastic normal
 * strain opening the crack).  The paper gives no formula for w_alpha; the reading used is the
 * inelastic part of the facet displacement jump: w_N = l <e_N - t_N / E0>, w_M = l (e_M - t_M / (alpha
 * E0)), w_L = l (e_L - t_L / (alpha E0)).  Also the volumetric strain of every tetrahedron (the field
 * the paper compares for the uniaxial-strain test).  Both at the current state. */
void orc_metrics(const orc_model *M, double *w, double *eV)
{
    if (w)
        for (int32_t k = 0; k < M->F; ++k) {
            const double E0 = M->pE0 ? M->pE0[k] : M->mat.E0;
            const double aE = (M->palpha ? M->palpha[k] : M->mat.alpha) * E0;
            const double *e = M->e_prev + 3 * (size_t)k, *t = M->t_loc + 3 * (size_t)k;
            double wn = e[0] - t[0] / E0;
            if (wn < 0.0) wn = 0.0;
            double wm = e[1] - t[1] / aE, wl = e[2] - t[2] / aE;
            w[k] = M->len[k] * sqrt(wn * wn + wm * wm + wl * wl);
        }
    if (eV)
        for (int32_t t = 0; t < M->T; ++t) eV[t] = tet_volumetric_strain(M, M->q, t);
}

/* Replace the boundary conditions (mask, velocities, ramp) for the following steps.  Velocities of
 * newly fixed or prescribed DOFs take their constrained values at the current time. */
void orc_set_bc(orc_model *M, const int32_t *mask, const double *vel, double ramp_time)
{
    size_t n6 = 6 * (size_t)M->N;
    memcpy(M->bc_mask, mask, sizeof(int32_t) * n6);
    if (vel)
        memcpy(M->bc_vel, vel, sizeof(double) * n6);
    else
        memset(M->bc_vel, 0, sizeof(double) * n6);
    M->ramp_time = ramp_time;
    double t = (double)M->step * M->dt;
    for (size_t i = 0; i < n6; ++i) {
        if (M->bc_mask[i] == 1) M->v[i] = 0.0;
        if (M->bc_mask[i] == 2) M->v[i] = M->bc_vel[i] * ramp(M, t);
    }
}

/* Perturbation study (Sec. 5): q += dq on the free DOFs; the strain of the perturbed state becomes
 * the reference of the next increment (as in orc_set_state); velocities, tractions, e_max and the node
 * forces (built from the tractions) are kept. */
void orc_perturb(orc_model *M, const double *dq)
{
    size_t n6 = 6 * (size_t)M->N;
    for (size_t i = 0; i < n6; ++i)
        if (M->bc_mask[i] == 0) M->q[i] += dq[i];
    for (int32_t k = 0; k < M->F; ++k) facet_strain(M, M->q, k, M->e_prev + 3 * (size_t)k);
}

/* Per-facet E0, alpha and sigma_t ([F] each, facet order of the model); a null array restores the
 * material's value for every facet.  The stored tractions are kept: the parameters act from the
 * next step on. */
void orc_set_facet_params(orc_model *M, const double *E0, const double *alpha, const double *sigma_t)
{
    double **dst[3] = {&M->pE0, &M->palpha, &M->psig};
    const double *src[3] = {E0, alpha, sigma_t};
    for (int i = 0; i < 3; ++i) {
        free(*dst[i]);
        *dst[i] = NULL;
        if (src[i]) {
            *dst[i] = (double *)malloc(sizeof(double) * M->F);
            memcpy(*dst[i], src[i], sizeof(double) * M->F);
        }
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Derivatives.                                                                                 */
/* ------------------------------------------------------------------------------------------ */

/* Jacobian of the constitutive update.  in = (e[3], de[3], eV, t_old[3], e_max_old, E0, alpha,
 * sigma_t); out = (t_new[3], e_max_new); jac[r * 14 + c] = d out[r] / d in[c].  The other material
 * parameters are those of *p. */
void orc_facet_law_jacobian(const orc_material *p, double l, const double in[14], double out[4], double jac[56])
{
    typedef Dual<14> S;
    S x[14];
    for (int c = 0; c < 14; ++c) {
        x[c] = S(in[c]);
        x[c].d[c] = 1.0;
    }
    S tn[3], em;
    facet_law<S>(p, x[11], x[12], x[13], l, x, x + 3, x[6], x + 7, x[10], tn, &em);
    const S *o[4] = {&tn[0], &tn[1], &tn[2], &em};
    for (int r = 0; r < 4; ++r) {
        out[r] = o[r]->v;
        for (int c = 0; c < 14; ++c) jac[14 * r + c] = o[r]->d[c];
    }
}

/* Objective of the adjoint and its directional derivatives.  From the current state, `nsteps` steps
 * are run (the model itself is left unchanged) and
 *     J = (1 / nsteps) sum_{n = 1..nsteps} sum_{constrained DOF i} seed_i (f_ext + R)_i (t_n),
 * the time mean of the seeded reactions.  For each of the nd directions (dE0, dalpha, dsigma_t)[d][F]
 * of the per-facet parameters, dJ[d] is the derivative of J along it, carried by forward-mode dual
 * numbers through the same step code (eight directions per pass).  Returns 0, or -5 when the
 * trajectory became non-finite. */
/* One trajectory of orc_tangent in scalar type S (double, or a dual number carrying the directions
 * d0 .. d0 + width - 1). */
template <class S, int Wd>
static int tangent_pass(const orc_model *M, int64_t nsteps, const double *seed, int32_t d0, int32_t nd,
                        const double *dE0, const double *dalpha, const double *dsigma_t, double *J, double *dJ)
{
    const size_t n6 = 6 * (size_t)M->N, F = (size_t)M->F;
    std::vector<S> q(n6), v(n6), f(n6), t(3 * F), em(F), ep(3 * F), Ff(3 * F), E0(F), al(F), sg(F);
    for (size_t i = 0; i < n6; ++i) {
        q[i] = S(M->q[i]);
        v[i] = S(M->v[i]);
        f[i] = S(M->f_asm[i]);
    }
    for (size_t k = 0; k < F; ++k) {
        for (int a = 0; a < 3; ++a) {
            t[3 * k + a] = S(M->t_loc[3 * k + a]);
            ep[3 * k + a] = S(M->e_prev[3 * k + a]);
        }
        em[k] = S(M->emax[k]);
        E0[k] = S(M->pE0 ? M->pE0[k] : M->mat.E0);
        al[k] = S(M->palpha ? M->palpha[k] : M->mat.alpha);
        sg[k] = S(M->psig ? M->psig[k] : M->mat.sigma_t);
        if constexpr (Wd > 0) {
            for (int w = 0; w < Wd && d0 + w < nd; ++w) {
                const size_t row = (size_t)(d0 + w) * F + k;
                if (dE0) E0[k].d[w] = dE0[row];
                if (dalpha) al[k].d[w] = dalpha[row];
                if (dsigma_t) sg[k].d[w] = dsigma_t[row];
            }
        }
    }
    Traj<S> T{q.data(), v.data(), f.data(), t.data(), em.data(), ep.data(), Ff.data(), E0.data(), al.data(), sg.data()};
    int64_t step = M->step;
    S Js(0.0);
    run_steps<S>(M, T, nsteps, &step, NULL, seed, &Js);
    int rc = 0;
    for (size_t i = 0; i < n6; ++i)
        if (!isfinite(value_of(q[i])) || !isfinite(value_of(v[i]))) rc = -5;
    const double inv = nsteps > 0 ? 1.0 / (double)nsteps : 0.0;
    if (J) *J = value_of(Js) * inv;
    if constexpr (Wd > 0) {
        for (int w = 0; w < Wd && d0 + w < nd; ++w)
            if (dJ) dJ[d0 + w] = Js.d[w] * inv;
    }
    return rc;
}

int orc_tangent(const orc_model *M, int64_t nsteps, const double *seed, int32_t nd, const double *dE0,
                const double *dalpha, const double *dsigma_t, double *J, double *dJ)
{
    if (nd <= 0) return tangent_pass<double, 0>(M, nsteps, seed, 0, 0, NULL, NULL, NULL, J, NULL);
    int rc = 0;
    for (int32_t d0 = 0; d0 < nd; d0 += 8) {
        int r = tangent_pass<Dual<8>, 8>(M, nsteps, seed, d0, nd, dE0, dalpha, dsigma_t, d0 == 0 ? J : NULL, dJ);
        if (r) rc = r;
    }
    return rc;
}
