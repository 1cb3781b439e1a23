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
 * Two variants of the composition scheme, both named in Sec. 3.3:
 *   - h_eq_alt = 1: the alternative equilibrium of Eq. Seq_Concent_Alt with
 *     H_k = 0 (Eq. LBE_Concent_Alt): h^eq,alt_k = w_k [gamma D mu + e_k.F / xi_s^2]
 *     for k != 0 (xi_s^2 = 1/3 in lattice units), h^eq,alt_0 = h^eq_0, and
 *     h*_k = h_k - (h_k - h^eq,alt_k) / (tau_h + 1/2).  Without H there is no
 *     shifted variable: the populations start at h_k = h^eq,alt_k (dphi/dt = 0).
 *   - h_lattice = 1: h on the smaller lattice of the paper's code (Sec. 3.1),
 *     D2Q5 in 2-D and D3Q7 in 3-D, with weights chosen so that xi_s^2 = 1/3 as
 *     for D2Q9 (tau_h = 3 dt / (gamma dx^2) unchanged): D2Q5 w = 1/3, 1/6;
 *     D3Q7 w = 0, 1/6.  g, the gradient and the normal keep D2Q9 / D3Q19.
 *
 * Unequal curvatures of the two parabolas (unequal_eps = 1, eps_ratio =
 * eps_s / eps_l, Sec. 2.3): with e_s = sqrt(eps_s / eps_l), e_l = 1 / e_s,
 *   closure (Eq. Closure, h = phi):
 *        mu = [c - phi m_l - (1 - phi) m_s] / [e_s phi + e_l (1 - phi)]
 *   S_phi (Eq. SourceTerm):
 *        S = p'(phi) [(e_l - e_s) mu^2 / 2 - (m_l - m_s) mu - df]
 *   anti-trapping (Eq. Anti-Trapping_Quadratic, coefficient a):
 *        j_at = a W [(e_l - e_s) mu + m_s - m_l] dphi n
 * The parameters stay the coexistence compositions and mu_eq; m_l, m_s and
 * df (Delta f^min) follow from the two equilibrium conditions of Sec. 2.3.2
 * (equal mu at c_s^co and c_l^co, equal grand potentials at mu_eq):
 *        m_l = c_l^co - e_s mu_eq,  m_s = c_s^co - e_l mu_eq,
 *        df = (e_l - e_s) mu_eq^2 / 2 - (m_l - m_s) mu_eq.
 * With eps_s = eps_l these reduce to the closure and sources above.
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
    int h_lattice;          /* 0: h on the g lattice; 1: D2Q5 / D3Q7 */
    int h_eq_alt;           /* 1: h^eq,alt with H = 0 (Eq. Seq_Concent_Alt) */
    int unequal_eps;        /* 1: parabolas of curvatures eps_s != eps_l */
    double eps_ratio;       /* eps_s / eps_l when unequal_eps = 1 */
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

/* D2Q5 (the first five D2Q9 directions) and D3Q7 (rest and the six face
 * links, opposites next to each other), for h only; weights with
 * xi_s^2 = sum_k w_k e_kx^2 = 1/3. */
static const double D2Q5_W[5] = {1.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0};
static const double D3Q7_W[7] = {0.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0};

typedef struct {
    int q;
    const int (*e)[3];
    const double *w;
    int opp[19];
} lattice;

static lattice make_lattice(int q, const int (*e)[3], const double *w)
{
    lattice L;
    L.q = q; L.e = e; L.w = w;
    for (int k = 0; k < L.q; ++k)
        for (int j = 0; j < L.q; ++j)
            if (L.e[j][0] == -L.e[k][0] && L.e[j][1] == -L.e[k][1] && L.e[j][2] == -L.e[k][2])
                L.opp[k] = j;
    return L;
}

static lattice get_lattice(int dim)
{
    return dim == 3 ? make_lattice(19, D3Q19_E, D3Q19_W) : make_lattice(9, D2Q9_E, D2Q9_W);
}

/* The lattice of the composition populations h. */
static lattice get_h_lattice(const or_params *p)
{
    if (!p->h_lattice) return get_lattice(p->dim);
    return p->dim == 3 ? make_lattice(7, D3Q19_E, D3Q7_W) : make_lattice(5, D2Q9_E, D2Q5_W);
}

/* Lattice tables, exported so that the tests can check the identities the
 * scheme relies on (sum w = 1, sum w e = 0, 3 sum w e e = I).  code: 2 D2Q9,
 * 3 D3Q19, 5 D2Q5, 7 D3Q7. */
int or_lattice(int code, int *e_out /* q*3 */, double *w_out /* q */, int *opp_out /* q */)
{
    lattice L;
    if (code == 5) L = make_lattice(5, D2Q9_E, D2Q5_W);
    else if (code == 7) L = make_lattice(7, D3Q19_E, D3Q7_W);
    else L = get_lattice(code);
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

/* Parabolas of unequal curvature: e_s, e_l, the minima m_s, m_l and df. */
typedef struct { double e_s, e_l, m_s, m_l, df; } parabolas;

static parabolas get_parabolas(const or_params *p)
{
    parabolas q;
    q.e_s = sqrt(p->eps_ratio);
    q.e_l = 1.0 / q.e_s;
    q.m_l = p->c_l_co - q.e_s * p->mu_eq;
    q.m_s = p->c_s_co - q.e_l * p->mu_eq;
    q.df = 0.5 * (q.e_l - q.e_s) * p->mu_eq * p->mu_eq - (q.m_l - q.m_s) * p->mu_eq;
    return q;
}

static double closure_mu(const or_params *p, double phi, double c)
{
    if (p->unequal_eps) {
        parabolas q = get_parabolas(p);
        return (c - phi * q.m_l - (1.0 - phi) * q.m_s) / (q.e_s * phi + q.e_l * (1.0 - phi));
    }
    /* h(phi) = phi, c^co(phi) = c_l^co h + c_s^co (1 - h) */
    double cco = p->c_l_co * phi + p->c_s_co * (1.0 - phi);
    return p->mu_eq + c - cco;
}

static double source_S(const or_params *p, double phi, double mu)
{
    double pprime = 6.0 * phi * (1.0 - phi);
    if (p->unequal_eps) {
        parabolas q = get_parabolas(p);
        return pprime * (0.5 * (q.e_l - q.e_s) * mu * mu - (q.m_l - q.m_s) * mu - q.df);
    }
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
    double jump = p->c_s_co - p->c_l_co;
    if (p->unequal_eps) {
        parabolas q = get_parabolas(p);
        jump = (q.e_l - q.e_s) * mu + q.m_s - q.m_l;
    }
    double at = p->anti_trapping ? p->a_at * p->W * jump * dphi : 0.0;
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

/* h^eq,alt of Eq. Seq_Concent_Alt: the flux enters the equilibrium through its
 * first moment, e_k.F / xi_s^2 with xi_s^2 = 1/3, and H_k = 0. */
static double h_equilibrium_alt(const or_params *p, const lattice *L, int k,
                                double phi, double c, double mu, const double F[3])
{
    double heq = h_equilibrium(p, L, k, phi, c, mu);
    if (k == 0) return heq;
    double eF = L->e[k][0] * F[0] + L->e[k][1] * F[1] + L->e[k][2] * F[2];
    return heq + L->w[k] * eF / (1.0 / 3.0);
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
    lattice LH = get_h_lattice(p);
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
            }
            for (int k = 0; k < LH.q; ++k) {
                if (p->h_eq_alt) {
                    h[k * N + i] = h_equilibrium_alt(p, &LH, k, phi[i], c[i], mu, F);
                } else {
                    double Hk = source_H(p, &LH, k, F);
                    h[k * N + i] = h_equilibrium(p, &LH, k, phi[i], c[i], mu) - 0.5 * Hk;
                }
            }
        }
    }
    return 0;
}

/* ---- one time step ----------------------------------------------------- */

static int step_once(const or_params *p, const lattice *L, const lattice *LH, double *g, double *h,
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
            for (int k = 0; k < LH->q; ++k) {
                if (p->h_eq_alt) {
                    double heq = h_equilibrium_alt(p, LH, k, phi[i], c[i], mu[i], F);
                    hs[k * N + i] = h[k * N + i] - omh * (h[k * N + i] - heq);
                } else {
                    double Hk = source_H(p, LH, k, F);
                    double heq_tilde = h_equilibrium(p, LH, k, phi[i], c[i], mu[i]) - 0.5 * Hk;
                    hs[k * N + i] = h[k * N + i] - omh * (h[k * N + i] - heq_tilde) + Hk;
                }
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
            for (int k = 0; k < LH->q; ++k) {
                long src = upstream_index(p, LH, k, x, y, z);
                double v = (src < 0) ? hs[LH->opp[k] * N + i] : hs[k * N + src];
                h[k * N + i] = v;
                s += v;
            }
            c[i] = s;
            phi[i] = phinew[i];
        }
    }
    return 0;
}

/* Advance nsteps.  h holds q_h planes (9 / 19, or 5 / 7 with h_lattice = 1).
 * Returns 0, or -1 on allocation failure. */
int or_step(const or_params *p, double *g, double *h, double *phi, double *c, int nsteps)
{
    lattice L = get_lattice(p->dim);
    lattice LH = get_h_lattice(p);
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
        rc = step_once(p, &L, &LH, g, h, phi, c, gs, hs, mu, grad, nvec, Gsum, phinew);
    free(gs); free(hs); free(mu); free(grad); free(nvec); free(Gsum); free(phinew);
    return rc;
}

/* mu from the closure, for reporting. */
void or_mu(const or_params *p, const double *phi, const double *c, double *mu)
{
    long N = (long)p->nx * p->ny * p->nz;
    for (long i = 0; i < N; ++i) mu[i] = closure_mu(p, phi[i], c[i]);
}

/* ======================================================================== */
/* Discrete adjoint (reverse mode) of one step and of the initialisation.    */
/*                                                                          */
/* The step is linear in the populations and a smooth function of phi and c; */
/* its adjoint is the chain rule taken back through the operations listed at */
/* the top of this file, in reverse order.  Parameters differentiated:       */
/* pb[0] = d/dD_l, pb[1] = d/dtau_g, pb[2] = d/dtau_h, pb[3] = d/dlambda,     */
/* with W, D_s, the coexistence values, a of j_at and eps_s / eps_l held     */
/* fixed.  It covers every option of the step (h on D2Q5 / D3Q7, h^eq,alt,  */
/* unequal curvatures).                                                      */
/* ======================================================================== */
#ifndef ORACLE_TANGENT_BUILD

/* Node that consumes the post-collision population j of node (x,y,z) when it
 * streams: x + e_j (wrapped), or -1 when x + e_j lies beyond a bounce-back wall
 * (the population then returns to the node itself as direction opp(j)). */
static long downstream_index(const or_params *p, const lattice *L, int j, int x, int y, int z)
{
    int n[3] = {p->nx, p->ny, p->nz};
    int c[3] = {x + L->e[j][0], y + L->e[j][1], z + L->e[j][2]};
    for (int a = 0; a < 3; ++a) {
        if (c[a] < 0 || c[a] >= n[a]) {
            if (p->bc[a] == 1) return -1;
            c[a] = wrap(c[a], n[a]);
        }
    }
    return idx(p, c[0], c[1], c[2]);
}

/* Adjoint of the pointwise sources at one node.  Given the adjoints Gb[j] of the
 * phi sources G_j (links of L), heqb[j] of the equilibria h^eq_j and Hb[j] of the
 * flux terms of the h collision (links of LH: H_j = gamma w_j e_j.F, or
 * A_j = w_j e_j.F / xi_s^2 of h^eq,alt), add the adjoints of phi, mu, n, grad,
 * dphi and of the parameters.  (Forward: Sec. 2.3, 3.2 and 3.3 formulas above.) */
static void pointwise_adjoint(const or_params *p, const lattice *L, const lattice *LH, double phi, double c,
                              double mu, double dphi, const double grad[3], const double nvec[3],
                              const double *Gb, const double *heqb, const double *Hb,
                              double *phib, double *mub, double gradb[3], double nb[3], double *cb,
                              double *dphib, double *pb)
{
    int q = L->q;
    double M = p->tau_g / 3.0;
    double W2 = p->W * p->W;
    double dc = p->c_s_co - p->c_l_co;
    double gamma = 3.0 / p->tau_h;
    double D = p->D_l * phi + p->D_s * (1.0 - phi);
    double Dprime = p->D_l - p->D_s;
    /* S = p'(phi) drive(mu), jump(mu) = coefficient of a W dphi n in j_at, and
     * their mu-derivatives (Eq. SourceTerm_Coexistence / Eq. SourceTerm;
     * Eq. Anti-trapping_Equilibrium / Eq. Anti-Trapping_Quadratic) */
    double drive = dc * (mu - p->mu_eq), drive_mu = dc, jump = dc, jump_mu = 0.0;
    if (p->unequal_eps) {
        parabolas pq = get_parabolas(p);
        drive = 0.5 * (pq.e_l - pq.e_s) * mu * mu - (pq.m_l - pq.m_s) * mu - pq.df;
        drive_mu = (pq.e_l - pq.e_s) * mu - (pq.m_l - pq.m_s);
        jump = (pq.e_l - pq.e_s) * mu + pq.m_s - pq.m_l;
        jump_mu = pq.e_l - pq.e_s;
    }

    /* G_j = w_j (Gst + Gcurv_j) */
    double Gstb = 0.0;
    for (int j = 0; j < q; ++j) Gstb += L->w[j] * Gb[j];
    double S = 6.0 * phi * (1.0 - phi) * drive;
    double Sb = Gstb * (-p->lambda * M / W2);
    pb[3] += Gstb * (-M * S / W2);
    pb[1] += Gstb * (-p->lambda * S / W2) / 3.0;
    *phib += Sb * 6.0 * (1.0 - 2.0 * phi) * drive;
    *mub += Sb * 6.0 * phi * (1.0 - phi) * drive_mu;
    if (p->counter_term) {
        double K = (4.0 / p->W) * phi * (1.0 - phi);
        double Kb = 0.0;
        for (int j = 0; j < q; ++j) {
            double en = L->e[j][0] * nvec[0] + L->e[j][1] * nvec[1] + L->e[j][2] * nvec[2];
            Kb += L->w[j] * en * Gb[j];
            for (int a = 0; a < 3; ++a) nb[a] += K * L->w[j] * L->e[j][a] * Gb[j];
        }
        *phib += Kb * (4.0 / p->W) * (1.0 - 2.0 * phi);
    } else {
        double wp = 2.0 * phi * (1.0 - phi) * (1.0 - 2.0 * phi);
        double wpp = 2.0 - 12.0 * phi + 12.0 * phi * phi;
        double Gcb = 0.0;
        for (int j = 0; j < q; ++j) Gcb += L->w[j] * Gb[j];
        *phib += Gcb * (-(8.0 * M / W2)) * wpp;
        pb[1] += Gcb * (-(8.0 / W2)) * wp / 3.0;
    }

    /* h^eq_0 = c - (1 - w_0) gamma D mu, h^eq_k = w_k gamma D mu (on LH) */
    int qh = LH->q;
    double Qb = -(1.0 - LH->w[0]) * heqb[0];
    *cb += heqb[0];
    for (int k = 1; k < qh; ++k) Qb += LH->w[k] * heqb[k];
    double gammab = Qb * D * mu;
    double Db = Qb * gamma * mu;
    *mub += Qb * gamma * D;
    *phib += Db * Dprime;
    pb[0] += Db * phi;

    /* H_k = gamma w_k e_k.F (or A_k = 3 w_k e_k.F with h^eq,alt),
     * F = mu D' grad + at n, at = s a W jump(mu) dphi */
    double F[3];
    double at = p->anti_trapping ? p->a_at * p->W * jump * dphi : 0.0;
    for (int a = 0; a < 3; ++a) F[a] = mu * Dprime * grad[a] + at * nvec[a];
    double Fb[3] = {0.0, 0.0, 0.0};
    double kF = p->h_eq_alt ? 3.0 : gamma;
    for (int k = 0; k < qh; ++k) {
        double eF = LH->e[k][0] * F[0] + LH->e[k][1] * F[1] + LH->e[k][2] * F[2];
        if (!p->h_eq_alt) gammab += LH->w[k] * eF * Hb[k];
        for (int a = 0; a < 3; ++a) Fb[a] += kF * LH->w[k] * LH->e[k][a] * Hb[k];
    }
    double Fg = Fb[0] * grad[0] + Fb[1] * grad[1] + Fb[2] * grad[2];
    double Fn = Fb[0] * nvec[0] + Fb[1] * nvec[1] + Fb[2] * nvec[2];
    *mub += Dprime * Fg;
    pb[0] += mu * Fg;
    for (int a = 0; a < 3; ++a) {
        gradb[a] += mu * Dprime * Fb[a];
        nb[a] += at * Fb[a];
    }
    if (p->anti_trapping) {
        *dphib += p->a_at * p->W * jump * Fn;
        *mub += p->a_at * p->W * jump_mu * dphi * Fn;
    }
    pb[2] += gammab * (-3.0 / (p->tau_h * p->tau_h));
}

/* Adjoint of the unit normal and of the closure, then the transpose of the
 * gradient stencil: the last three operations of every node, reversed. */
static void finish_adjoint(const or_params *p, const lattice *L, const double *phi, const double *mu,
                           const double *grad, const double *nvec,
                           double *gradb, double *nb, double *mub, double *phib, double *cb)
{
    long N = (long)p->nx * p->ny * p->nz;
    for (long i = 0; i < N; ++i) {
        const double *gr = grad + 3 * i, *nv = nvec + 3 * i;
        double g2 = gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2];
        double inv = 1.0 / sqrt(g2 + p->eps_n * p->eps_n);
        double nn = nv[0] * nb[3 * i] + nv[1] * nb[3 * i + 1] + nv[2] * nb[3 * i + 2];
        for (int a = 0; a < 3; ++a) gradb[3 * i + a] += (nb[3 * i + a] - nv[a] * nn) * inv;
        if (p->unequal_eps) {
            /* mu = [c - phi m_l - (1 - phi) m_s] / den, den = e_s phi + e_l (1 - phi) */
            parabolas pq = get_parabolas(p);
            double den = pq.e_s * phi[i] + pq.e_l * (1.0 - phi[i]);
            cb[i] += mub[i] / den;
            phib[i] += mub[i] * (-(pq.m_l - pq.m_s) - mu[i] * (pq.e_s - pq.e_l)) / den;
        } else {
            cb[i] += mub[i];
            phib[i] += mub[i] * (p->c_s_co - p->c_l_co);
        }
    }
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long i = idx(p, x, y, z);
                for (int k = 1; k < L->q; ++k) {
                    const int *e = L->e[k];
                    double t = 1.5 * L->w[k] * (e[0] * gradb[3 * i] + e[1] * gradb[3 * i + 1] + e[2] * gradb[3 * i + 2]);
                    phib[stencil_index(p, x + e[0], y + e[1], z + e[2])] += t;
                    phib[stencil_index(p, x - e[0], y - e[1], z - e[2])] -= t;
                }
            }
}

/* Adjoint of one step.  (g, h, phi, c): the state at step n.  On entry gb, hb,
 * phib, cb hold the adjoints of the state at step n+1; on return they hold the
 * adjoints of the state at step n.  pb[4] accumulates the parameter adjoints.
 * Returns 0, or -1 on allocation failure. */
int or_step_adjoint(const or_params *p, const double *g, const double *h, const double *phi, const double *c,
                    double *gb, double *hb, double *phib, double *cb, double *pb)
{
    lattice L = get_lattice(p->dim);
    lattice LH = get_h_lattice(p);
    long N = (long)p->nx * p->ny * p->nz;
    int q = L.q, qh = LH.q;
    double omg = 1.0 / (p->tau_g + 0.5), omh = 1.0 / (p->tau_h + 0.5);
    double *mu = malloc(sizeof(double) * N), *grad = malloc(sizeof(double) * 3 * N);
    double *nvec = malloc(sizeof(double) * 3 * N), *gs = malloc(sizeof(double) * q * N);
    double *phinew = malloc(sizeof(double) * N), *Gsum = malloc(sizeof(double) * N);
    double *gbo = malloc(sizeof(double) * q * N), *hbo = malloc(sizeof(double) * qh * N);
    double *phibo = calloc(N, sizeof(double)), *cbo = calloc(N, sizeof(double));
    double *mub = calloc(N, sizeof(double)), *gradb = calloc(3 * N, sizeof(double));
    double *nb = calloc(3 * N, sizeof(double)), *dphib = calloc(N, sizeof(double));
    int rc = 0;
    if (!mu || !grad || !nvec || !gs || !phinew || !Gsum || !gbo || !hbo || !phibo || !cbo || !mub || !gradb ||
        !nb || !dphib) rc = -1;
    if (rc == 0) {
        /* forward recomputation of the step's intermediates */
        for (int z = 0; z < p->nz; ++z)
            for (int y = 0; y < p->ny; ++y)
                for (int x = 0; x < p->nx; ++x) {
                    long i = idx(p, x, y, z);
                    mu[i] = closure_mu(p, phi[i], c[i]);
                    gradient_at(p, &L, phi, x, y, z, grad + 3 * i);
                    normal_from(p, grad + 3 * i, nvec + 3 * i);
                    double s = 0.0;
                    for (int k = 0; k < q; ++k) {
                        double Gk = source_G(p, &L, k, phi[i], mu[i], nvec + 3 * i);
                        double geq_tilde = L.w[k] * phi[i] - 0.5 * Gk;
                        gs[k * N + i] = g[k * N + i] - omg * (g[k * N + i] - geq_tilde) + Gk;
                        s += Gk;
                    }
                    Gsum[i] = s;
                }
        for (int z = 0; z < p->nz; ++z)
            for (int y = 0; y < p->ny; ++y)
                for (int x = 0; x < p->nx; ++x) {
                    long i = idx(p, x, y, z);
                    double s = 0.0;
                    for (int k = 0; k < q; ++k) {
                        long src = upstream_index(p, &L, k, x, y, z);
                        s += (src < 0) ? gs[L.opp[k] * N + i] : gs[k * N + src];
                    }
                    phinew[i] = s + 0.5 * Gsum[i];
                }
        /* composition part, reversed: c' = sum h', stream, collision, sources */
        for (int z = 0; z < p->nz; ++z)
            for (int y = 0; y < p->ny; ++y)
                for (int x = 0; x < p->nx; ++x) {
                    long i = idx(p, x, y, z);
                    double dphi = phinew[i] - phi[i];
                    double hsb[19], heqb[19], Hb[19], Gb0[19];
                    double F[3];
                    flux_F(p, mu[i], dphi, grad + 3 * i, nvec + 3 * i, F);
                    double omhb = 0.0;
                    for (int j = 0; j < q; ++j) Gb0[j] = 0.0;
                    for (int j = 0; j < qh; ++j) {
                        long y2 = downstream_index(p, &LH, j, x, y, z);
                        hsb[j] = (y2 < 0) ? hb[LH.opp[j] * N + i] + cb[i] : hb[j * N + y2] + cb[y2];
                        hbo[j * N + i] = (1.0 - omh) * hsb[j];
                        heqb[j] = omh * hsb[j];
                        if (p->h_eq_alt) {
                            /* h* = h - omh (h - h^eq,alt): the flux part A_j enters with omh */
                            double heq = h_equilibrium_alt(p, &LH, j, phi[i], c[i], mu[i], F);
                            Hb[j] = omh * hsb[j];
                            omhb += hsb[j] * (heq - h[j * N + i]);
                        } else {
                            double Hj = source_H(p, &LH, j, F);
                            double heq = h_equilibrium(p, &LH, j, phi[i], c[i], mu[i]);
                            Hb[j] = (1.0 - 0.5 * omh) * hsb[j];
                            omhb += hsb[j] * (heq - 0.5 * Hj - h[j * N + i]);
                        }
                    }
                    pb[2] += omhb * (-omh * omh);
                    pointwise_adjoint(p, &L, &LH, phi[i], c[i], mu[i], dphi, grad + 3 * i, nvec + 3 * i, Gb0, heqb,
                                      Hb, phibo + i, mub + i, gradb + 3 * i, nb + 3 * i, cbo + i, dphib + i, pb);
                }
        /* phi part, reversed: phi' = sum g' + G/2, stream, collision, sources */
        for (int z = 0; z < p->nz; ++z)
            for (int y = 0; y < p->ny; ++y)
                for (int x = 0; x < p->nx; ++x) {
                    long i = idx(p, x, y, z);
                    double Gb[19], zero[19], dummy = 0.0;
                    double omgb = 0.0, phinewb_here = phib[i] + dphib[i];
                    for (int j = 0; j < q; ++j) {
                        long y2 = downstream_index(p, &L, j, x, y, z);
                        double gsb = (y2 < 0) ? gb[L.opp[j] * N + i] + phinewb_here
                                              : gb[j * N + y2] + phib[y2] + dphib[y2];
                        double Gj = source_G(p, &L, j, phi[i], mu[i], nvec + 3 * i);
                        gbo[j * N + i] = (1.0 - omg) * gsb;
                        phibo[i] += omg * L.w[j] * gsb;
                        Gb[j] = (1.0 - 0.5 * omg) * gsb + 0.5 * phinewb_here;
                        omgb += gsb * (L.w[j] * phi[i] - 0.5 * Gj - g[j * N + i]);
                        zero[j] = 0.0;
                    }
                    pb[1] += omgb * (-omg * omg);
                    phibo[i] -= dphib[i];                 /* dphi = phi' - phi */
                    for (int j = q; j < 19; ++j) zero[j] = 0.0;
                    pointwise_adjoint(p, &L, &LH, phi[i], c[i], mu[i], 0.0, grad + 3 * i, nvec + 3 * i, Gb, zero,
                                      zero, phibo + i, mub + i, gradb + 3 * i, nb + 3 * i, cbo + i, &dummy, pb);
                }
        finish_adjoint(p, &L, phi, mu, grad, nvec, gradb, nb, mub, phibo, cbo);
        memcpy(gb, gbo, sizeof(double) * q * N);
        memcpy(hb, hbo, sizeof(double) * qh * N);
        memcpy(phib, phibo, sizeof(double) * N);
        memcpy(cb, cbo, sizeof(double) * N);
    }
    free(mu); free(grad); free(nvec); free(gs); free(phinew); free(Gsum); free(gbo); free(hbo);
    free(phibo); free(cbo); free(mub); free(gradb); free(nb); free(dphib);
    return rc;
}

/* Adjoint of or_init.  On entry gb, hb hold the adjoints of the initial
 * populations and phib, cb those of the initial fields; on return phib, cb
 * hold the adjoints of phi0 and c0.  pb[4] accumulates the parameter adjoints. */
int or_init_adjoint(const or_params *p, const double *phi0, const double *c0, const double *gb, const double *hb,
                    double *phib, double *cb, double *pb)
{
    lattice L = get_lattice(p->dim);
    lattice LH = get_h_lattice(p);
    long N = (long)p->nx * p->ny * p->nz;
    int q = L.q, qh = LH.q;
    double *mu = malloc(sizeof(double) * N), *grad = malloc(sizeof(double) * 3 * N);
    double *nvec = malloc(sizeof(double) * 3 * N), *mub = calloc(N, sizeof(double));
    double *gradb = calloc(3 * N, sizeof(double)), *nb = calloc(3 * N, sizeof(double));
    int rc = (mu && grad && nvec && mub && gradb && nb) ? 0 : -1;
    if (rc == 0) {
        for (int z = 0; z < p->nz; ++z)
            for (int y = 0; y < p->ny; ++y)
                for (int x = 0; x < p->nx; ++x) {
                    long i = idx(p, x, y, z);
                    mu[i] = closure_mu(p, phi0[i], c0[i]);
                    gradient_at(p, &L, phi0, x, y, z, grad + 3 * i);
                    normal_from(p, grad + 3 * i, nvec + 3 * i);
                }
        for (long i = 0; i < N; ++i) {
            /* g_k = w_k phi0 - G_k/2;  h_k = h^eq_k - H_k/2 with dphi/dt = 0, or
             * h_k = h^eq_k + A_k (h^eq,alt) */
            double Gb[19], heqb[19], Hb[19], dummy = 0.0;
            for (int j = 0; j < q; ++j) {
                phib[i] += L.w[j] * gb[j * N + i];
                Gb[j] = -0.5 * gb[j * N + i];
            }
            for (int j = 0; j < qh; ++j) {
                heqb[j] = hb[j * N + i];
                Hb[j] = (p->h_eq_alt ? 1.0 : -0.5) * hb[j * N + i];
            }
            pointwise_adjoint(p, &L, &LH, phi0[i], c0[i], mu[i], 0.0, grad + 3 * i, nvec + 3 * i, Gb, heqb, Hb,
                              phib + i, mub + i, gradb + 3 * i, nb + 3 * i, cb + i, &dummy, pb);
        }
        finish_adjoint(p, &L, phi0, mu, grad, nvec, gradb, nb, mub, phib, cb);
    }
    free(mu); free(grad); free(nvec); free(mub); free(gradb); free(nb);
    return rc;
}
#endif /* ORACLE_TANGENT_BUILD */
