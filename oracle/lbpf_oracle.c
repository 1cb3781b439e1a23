/*
 * FP64 CPU oracle of the coupled phi-mu lattice Boltzmann time step of
 * Boutin, Verdier & Cartalade, "Grand-potential-based phase-field model of
 * dissolution/precipitation" (arXiv 2111.05960).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only the tests, the smoke check and the timed CPU baseline
 * of the benchmark use it.  It shares no code, header, table or helper with
 * the CUDA library.
 *
 * Every quantity is in lattice units (dx = dt = 1, so xi_k = e_k and
 * xi_s^2 = 1/3).  Each step follows the paper's order of operations:
 *
 *   1. closure (Eq. PotChim_Equilibirum, Eq. Coexistence_Interpol, h = phi):
 *        mu = mu_eq + c - [c_l^co phi + c_s^co (1 - phi)]
 *   2. directional derivatives and gradient (Eq. DerivDirec_Grad, Eq. Grad):
 *        d_k = [phi(x+e_k) - phi(x-e_k)] / 2,  grad = 3 sum_k w_k e_k d_k
 *      unit normal (Eq. NormalVector), regularised: n = grad/sqrt(|grad|^2+eps^2)
 *   3. phi source (Eq. TermG, SourceG_ST, SourceG_dw, SourceG_CT; Tab. 2):
 *        S = p'(phi) (c_s^co - c_l^co)(mu - mu_eq),  p' = 6 phi (1-phi)
 *        G^st = -lambda M S / W^2,  M = tau_g / 3
 *        counter term on : G_k = w_k [G^st + (4/W) phi(1-phi) e_k.n]
 *        counter term off: G_k = w_k [G^st - (8M/W^2) omega'(phi)],
 *                          omega' = 2 phi (1-phi)(1-2 phi)
 *   4. g collision (Eq. LBE_PhaseField_Eq, Geq_Allen-Cahn_Eq-1):
 *        g*_k = g_k - (g_k - (w_k phi - G_k/2)) / (tau_g + 1/2) + G_k
 *   5. streaming g_k(x, n+1) = g*_k(x - e_k), half-way bounce-back at walls
 *   6. phi moment (Eq. Moment_Phi): phi' = sum_k g_k(x,n+1) + 1/2 sum_k G_k(x)
 *      time derivative by explicit Euler: dphi = phi' - phi
 *   7. c source (Eq. Anti-trapping_Equilibrium, Eq. SourceTerm_LBE_h):
 *        D = D_l phi + D_s (1 - phi),  D' = D_l - D_s
 *        j_at = a W (c_s^co - c_l^co) dphi n      (only when anti-trapping is on)
 *        F = mu D' grad + j_at,  gamma = 3 / tau_h,  H_k = gamma w_k e_k.F
 *   8. c equilibrium and collision (Eq. Heq_Composition, Eq. LBE_Composition):
 *        h^eq_0 = c - (1 - w_0) gamma D mu,  h^eq_k = w_k gamma D mu  (k != 0)
 *        h*_k = h_k - (h_k - (h^eq_k - H_k/2)) / (tau_h + 1/2) + H_k
 *   9. streaming of h as for g, c' = sum_k h_k (Eq. Moment0_LBM_Concent)
 *
 * Lattices: D2Q9 in the paper's ordering (Sec. 3.1); D3Q19 for the 3-D
 * workloads (the paper names D3Q19 among the lattices of its code, Sec. 3.1),
 * with the same directional-derivative gradient over its 18 links.
 *
 * Boundaries: periodic, or half-way bounce-back (the wall sits half a cell
 * outside the first and last node): a population whose upstream node lies
 * outside the domain is replaced by the post-collision population of the
 * opposite direction at the node itself.  The phi stencil uses mirror ghosts
 * across a wall, phi(-1) = phi(0), phi(-2) = phi(1) (zero normal gradient).
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC.  No FMA
 * contraction, so every product and sum rounds as written.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int dim;                /* 2 or 3 */
    int nx, ny, nz;         /* nz = 1 in 2-D */
    int bc[3];              /* per axis: 0 periodic, 1 half-way bounce-back */
    double tau_g, tau_h;    /* dimensionless relaxation times */
    double W, lambda, D_l, D_s;
    double c_s_co, c_l_co, mu_eq;
    int counter_term;       /* 1: G^ct, 0: G^dw */
    int anti_trapping;      /* 1: j_at included */
    double a_at;            /* coefficient a of j_at */
    double eps_n;           /* regularisation of |grad phi| in n */
} or_params;

/* ---- lattices ---------------------------------------------------------- */

/* D2Q9, Sec. 3.1: e0 = 0, e1..e4 = (1,0),(0,1),(-1,0),(0,-1),
 * e5..e8 = (1,1),(-1,1),(-1,-1),(1,-1); w = 4/9, 1/9, 1/36. */
static const int D2Q9_E[9][3] = {
    {0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0},
    {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
static const double D2Q9_W[9] = {
    4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

/* D3Q19: rest, 6 face links (w = 1/18), 12 edge links (w = 1/36).  Opposite
 * directions sit next to each other (1<->2, 3<->4, ...). */
static const int D3Q19_E[19][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static const double D3Q19_W[19] = {
    1.0 / 3.0,
    1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

typedef struct {
    int q;
    const int (*e)[3];
    const double *w;
    int opp[19];
} lattice;

static lattice get_lattice(int dim)
{
    lattice L;
    if (dim == 3) { L.q = 19; L.e = D3Q19_E; L.w = D3Q19_W; }
    else          { L.q = 9;  L.e = D2Q9_E;  L.w = D2Q9_W; }
    for (int k = 0; k < L.q; ++k)
        for (int j = 0; j < L.q; ++j)
            if (L.e[j][0] == -L.e[k][0] && L.e[j][1] == -L.e[k][1] && L.e[j][2] == -L.e[k][2])
                L.opp[k] = j;
    return L;
}

/* Lattice tables, exported so that the tests can check the identities the
 * scheme relies on (sum w = 1, sum w e = 0, 3 sum w e e = I). */
int or_lattice(int dim, int *e_out /* q*3 */, double *w_out /* q */, int *opp_out /* q */)
{
    lattice L = get_lattice(dim);
    for (int k = 0; k < L.q; ++k) {
        for (int a = 0; a < 3; ++a) e_out[3 * k + a] = L.e[k][a];
        w_out[k] = L.w[k];
        opp_out[k] = L.opp[k];
    }
    return L.q;
}

/* ---- indexing ---------------------------------------------------------- */

static long idx(const or_params *p, int x, int y, int z)
{
    return ((long)z * p->ny + y) * p->nx + x;
}

static int wrap(int i, int n) { return ((i % n) + n) % n; }

/* Index of a node for the phi stencil: periodic wrap, or mirror ghost across
 * a bounce-back wall (phi(-1) = phi(0), phi(n) = phi(n-1), ...). */
static int ghost(int i, int n, int bc)
{
    if (bc == 0) return wrap(i, n);
    while (i < 0 || i >= n) {
        if (i < 0) i = -1 - i;
        if (i >= n) i = 2 * n - 1 - i;
    }
    return i;
}

static long stencil_index(const or_params *p, int x, int y, int z)
{
    int n[3] = {p->nx, p->ny, p->nz};
    int c[3] = {x, y, z};
    for (int a = 0; a < 3; ++a) c[a] = ghost(c[a], n[a], p->bc[a]);
    return idx(p, c[0], c[1], c[2]);
}

/* Upstream node of a pull along e_k; returns -1 when it lies beyond a
 * bounce-back wall. */
static long upstream_index(const or_params *p, const lattice *L, int k, int x, int y, int z)
{
    int n[3] = {p->nx, p->ny, p->nz};
    int c[3] = {x - L->e[k][0], y - L->e[k][1], z - L->e[k][2]};
    for (int a = 0; a < 3; ++a) {
        if (c[a] < 0 || c[a] >= n[a]) {
            if (p->bc[a] == 1) return -1;
            c[a] = wrap(c[a], n[a]);
        }
    }
    return idx(p, c[0], c[1], c[2]);
}

/* ---- pointwise model functions (Tab. 2 and Sec. 2.3) ------------------ */

static double closure_mu(const or_params *p, double phi, double c)
{
    /* h(phi) = phi, c^co(phi) = c_l^co h + c_s^co (1 - h) */
    double cco = p->c_l_co * phi + p->c_s_co * (1.0 - phi);
    return p->mu_eq + c - cco;
}

static double source_S(const or_params *p, double phi, double mu)
{
    double pprime = 6.0 * phi * (1.0 - phi);
    return pprime * (p->c_s_co - p->c_l_co) * (mu - p->mu_eq);
}

/* G_k of Eq. TermG at one node. */
static double source_G(const or_params *p, const lattice *L, int k,
                       double phi, double mu, const double nvec[3])
{
    double M = p->tau_g / 3.0;
    double Gst = -p->lambda * M * source_S(p, phi, mu) / (p->W * p->W);
    double Gcurv;
    if (p->counter_term) {
        double en = L->e[k][0] * nvec[0] + L->e[k][1] * nvec[1] + L->e[k][2] * nvec[2];
        Gcurv = (4.0 / p->W) * phi * (1.0 - phi) * en;
    } else {
        double wprime = 2.0 * phi * (1.0 - phi) * (1.0 - 2.0 * phi);
        Gcurv = -(8.0 * M / (p->W * p->W)) * wprime;
    }
    return L->w[k] * (Gst + Gcurv);
}

/* Flux F = mu D' grad(phi) + j_at of Eq. SourceTerm_LBE_h. */
static void flux_F(const or_params *p, double mu, double dphi,
                   const double grad[3], const double nvec[3], double F[3])
{
    double Dprime = p->D_l - p->D_s;
    double at = p->anti_trapping ? p->a_at * p->W * (p->c_s_co - p->c_l_co) * dphi : 0.0;
    for (int a = 0; a < 3; ++a) F[a] = mu * Dprime * grad[a] + at * nvec[a];
}

static double source_H(const or_params *p, const lattice *L, int k, const double F[3])
{
    double gamma = 3.0 / p->tau_h;
    double eF = L->e[k][0] * F[0] + L->e[k][1] * F[1] + L->e[k][2] * F[2];
    return gamma * L->w[k] * eF;
}

static double h_equilibrium(const or_params *p, const lattice *L, int k,
                            double phi, double c, double mu)
{
    double gamma = 3.0 / p->tau_h;
    double D = p->D_l * phi + p->D_s * (1.0 - phi);
    if (k == 0) return c - (1.0 - L->w[0]) * gamma * D * mu;
    return L->w[k] * gamma * D * mu;
}

/* Gradient by directional derivatives (Eq. DerivDirec_Grad and Eq. Grad). */
static void gradient_at(const or_params *p, const lattice *L, const double *phi,
                        int x, int y, int z, double grad[3])
{
    grad[0] = grad[1] = grad[2] = 0.0;
    for (int k = 1; k < L->q; ++k) {
        const int *e = L->e[k];
        double fwd = phi[stencil_index(p, x + e[0], y + e[1], z + e[2])];
        double bwd = phi[stencil_index(p, x - e[0], y - e[1], z - e[2])];
        double dk = 0.5 * (fwd - bwd);
        for (int a = 0; a < 3; ++a) grad[a] += 3.0 * L->w[k] * e[a] * dk;
    }
}

static void normal_from(const or_params *p, const double grad[3], double nvec[3])
{
    double g2 = grad[0] * grad[0] + grad[1] * grad[1] + grad[2] * grad[2];
    double inv = 1.0 / sqrt(g2 + p->eps_n * p->eps_n);
    for (int a = 0; a < 3; ++a) nvec[a] = grad[a] * inv;
}

/* Exported for the gradient pin: grad_out is [N][3]. */
void or_gradient(const or_params *p, const double *phi, double *grad_out)
{
    lattice L = get_lattice(p->dim);
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x)
                gradient_at(p, &L, phi, x, y, z, grad_out + 3 * idx(p, x, y, z));
}

/* ---- threads ----------------------------------------------------------- */

void or_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int or_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---- initialisation ---------------------------------------------------- */

/* g_k = g^eq_k - G_k/2 and h_k = h^eq_k - H_k/2 (the variable change of
 * Sec. 3.1 applied to populations at equilibrium), with H evaluated at
 * dphi/dt = 0.  Returns 0, or -1 on allocation failure. */
int or_init(const or_params *p, const double *phi0, const double *c0,
            double *g, double *h, double *phi, double *c)
{
    lattice L = get_lattice(p->dim);
    long N = (long)p->nx * p->ny * p->nz;
    memcpy(phi, phi0, sizeof(double) * N);
    memcpy(c, c0, sizeof(double) * N);
    long rows = (long)p->ny * p->nz;
#pragma omp parallel for schedule(static)
    for (long r = 0; r < rows; ++r) {
        int y = (int)(r % p->ny), z = (int)(r / p->ny);
        for (int x = 0; x < p->nx; ++x) {
            long i = idx(p, x, y, z);
            double grad[3], nvec[3], F[3];
            gradient_at(p, &L, phi, x, y, z, grad);
            normal_from(p, grad, nvec);
            double mu = closure_mu(p, phi[i], c[i]);
            flux_F(p, mu, 0.0, grad, nvec, F);
            for (int k = 0; k < L.q; ++k) {
                double Gk = source_G(p, &L, k, phi[i], mu, nvec);
                g[k * N + i] = L.w[k] * phi[i] - 0.5 * Gk;
                double Hk = source_H(p, &L, k, F);
                h[k * N + i] = h_equilibrium(p, &L, k, phi[i], c[i], mu) - 0.5 * Hk;
            }
        }
    }
    return 0;
}

/* ---- one time step ----------------------------------------------------- */

static int step_once(const or_params *p, const lattice *L, double *g, double *h,
                     double *phi, double *c, double *gs, double *hs,
                     double *mu, double *grad, double *nvec, double *Gsum, double *phinew)
{
    long N = (long)p->nx * p->ny * p->nz;
    long rows = (long)p->ny * p->nz;
    int q = L->q;
    double omg = 1.0 / (p->tau_g + 0.5);
    double omh = 1.0 / (p->tau_h + 0.5);

    /* 1-4: closure, gradient, normal, phi source and g collision */
#pragma omp parallel for schedule(static)
    for (long r = 0; r < rows; ++r) {
        int y = (int)(r % p->ny), z = (int)(r / p->ny);
        for (int x = 0; x < p->nx; ++x) {
            long i = idx(p, x, y, z);
            mu[i] = closure_mu(p, phi[i], c[i]);
            gradient_at(p, L, phi, x, y, z, grad + 3 * i);
            normal_from(p, grad + 3 * i, nvec + 3 * i);
            double sumG = 0.0;
            for (int k = 0; k < q; ++k) {
                double Gk = source_G(p, L, k, phi[i], mu[i], nvec + 3 * i);
                double geq_tilde = L->w[k] * phi[i] - 0.5 * Gk;
                gs[k * N + i] = g[k * N + i] - omg * (g[k * N + i] - geq_tilde) + Gk;
                sumG += Gk;
            }
            Gsum[i] = sumG;
        }
    }
    /* 5-6: stream g, new phi */
#pragma omp parallel for schedule(static)
    for (long r = 0; r < rows; ++r) {
        int y = (int)(r % p->ny), z = (int)(r / p->ny);
        for (int x = 0; x < p->nx; ++x) {
            long i = idx(p, x, y, z);
            double s = 0.0;
            for (int k = 0; k < q; ++k) {
                long src = upstream_index(p, L, k, x, y, z);
                double v = (src < 0) ? gs[L->opp[k] * N + i] : gs[k * N + src];
                g[k * N + i] = v;
                s += v;
            }
            phinew[i] = s + 0.5 * Gsum[i];
        }
    }
    /* 7-8: c source and h collision, with dphi = phi(n+1) - phi(n) */
#pragma omp parallel for schedule(static)
    for (long r = 0; r < rows; ++r) {
        int y = (int)(r % p->ny), z = (int)(r / p->ny);
        for (int x = 0; x < p->nx; ++x) {
            long i = idx(p, x, y, z);
            double dphi = phinew[i] - phi[i];
            double F[3];
            flux_F(p, mu[i], dphi, grad + 3 * i, nvec + 3 * i, F);
            for (int k = 0; k < q; ++k) {
                double Hk = source_H(p, L, k, F);
                double heq_tilde = h_equilibrium(p, L, k, phi[i], c[i], mu[i]) - 0.5 * Hk;
                hs[k * N + i] = h[k * N + i] - omh * (h[k * N + i] - heq_tilde) + Hk;
            }
        }
    }
    /* 9: stream h, new c; commit phi */
#pragma omp parallel for schedule(static)
    for (long r = 0; r < rows; ++r) {
        int y = (int)(r % p->ny), z = (int)(r / p->ny);
        for (int x = 0; x < p->nx; ++x) {
            long i = idx(p, x, y, z);
            double s = 0.0;
            for (int k = 0; k < q; ++k) {
                long src = upstream_index(p, L, k, x, y, z);
                double v = (src < 0) ? hs[L->opp[k] * N + i] : hs[k * N + src];
                h[k * N + i] = v;
                s += v;
            }
            c[i] = s;
            phi[i] = phinew[i];
        }
    }
    return 0;
}

/* Advance nsteps.  Returns 0, or -1 on allocation failure. */
int or_step(const or_params *p, double *g, double *h, double *phi, double *c, int nsteps)
{
    lattice L = get_lattice(p->dim);
    long N = (long)p->nx * p->ny * p->nz;
    int q = L.q;
    double *gs = malloc(sizeof(double) * q * N);
    double *hs = malloc(sizeof(double) * q * N);
    double *mu = malloc(sizeof(double) * N);
    double *grad = malloc(sizeof(double) * 3 * N);
    double *nvec = malloc(sizeof(double) * 3 * N);
    double *Gsum = malloc(sizeof(double) * N);
    double *phinew = malloc(sizeof(double) * N);
    int rc = 0;
    if (!gs || !hs || !mu || !grad || !nvec || !Gsum || !phinew) rc = -1;
    for (int s = 0; rc == 0 && s < nsteps; ++s)
        rc = step_once(p, &L, g, h, phi, c, gs, hs, mu, grad, nvec, Gsum, phinew);
    free(gs); free(hs); free(mu); free(grad); free(nvec); free(Gsum); free(phinew);
    return rc;
}

/* mu from the closure, for reporting. */
void or_mu(const or_params *p, const double *phi, const double *c, double *mu)
{
    long N = (long)p->nx * p->ny * p->nz;
    for (long i = 0; i < N; ++i) mu[i] = closure_mu(p, phi[i], c[i]);
}
