/*
 * vans_oracle.c -- plain FP64 CPU oracle of the porous (volume-averaged
 * Navier-Stokes) lattice Boltzmann model of Zhang, Wang & Ouyang,
 * "Lattice Boltzmann Model for the Volume-Averaged Navier-Stokes Equations".
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header, table or constant with the CUDA
 * library: the lattice tables below are written out here on their own.
 *
 * The oracle is the method written out step by step in double precision, in the
 * paper's order and notation, with no blocking, fusion or reordering:
 *
 *   state     f_i(x, t), the populations after streaming (the paper's f_i(x,t))
 *   moments   eps*rho = sum_i f_i                                  (Eq. 0moment)
 *             eps*rho*u = sum_i e_i f_i + dt/2 cs^2 rho grad(eps)
 *                         + dt/2 F                                  (Eq. 1moment)
 *   drag      F = -(eps^2 nu / K) u - (eps^3 F_eps / sqrt K) |u| u  (drag law,
 *             Sec. "Examples and discussions"), with the Ergun K and F_eps
 *   equilib.  f_i^eq = w_i eps rho [1 + e.u/cs^2 + (e.u)^2/(2cs^4)
 *                                   - u.u/(2cs^2)]                  (Eq. d2q9eq)
 *   sources   P_i = (1 - 1/(2tau)) w_i [(e_i-u)/cs^2 + (e_i.u) e_i/cs^4] . p grad eps
 *                                                                   (Eq. pi)
 *             F_i = (1 - 1/(2tau)) w_i [(e_i-u)/cs^2 + (e_i.u) e_i/cs^4] . F
 *                                                                   (Eq. Fi)
 *   update    f_i(x+e_i, t+1) = f_i - (f_i - f_i^eq)/tau + P_i + F_i
 *             (the final LBE with forcing, Sec. "Chapman-Enskog analysis")
 *
 * Readings of points the paper leaves open (each is stated where it is used):
 *   R1  D2Q9 / D3Q19 velocity sets and weights of Qian et al. (1992), cs^2 = 1/3.
 *   R2  Eq. d2q9eq's "e.u" is e_i.u.
 *   R3  F depends on u and Eq. 1moment is implicit in u.  |u|(a + b|u|) = |m| is a
 *       scalar quadratic, so u = 2m / (a + sqrt(a^2 + 4b|m|)) with
 *       m = sum e_i f_i + 1/2 cs^2 rho grad eps + 1/2 eps rho g,
 *       a = eps rho + alpha/2, b = beta/2 (exact, no iteration).
 *   R4  The drag carries no rho (as printed).  The driving body force is
 *       eps*rho*g (force per unit volume of the fluid phase) and is added to F.
 *   R5  grad eps = (1/cs^2) sum_i w_i e_i eps(x + e_i); a neighbour past a wall
 *       is replaced by eps(x); periodic axes wrap.
 *   R6  alpha = eps^2 nu / K and beta = eps^3 F_eps / sqrt(K) with the Ergun K
 *       and F_eps substituted are written as 150 nu (1-eps)^2 / (eps d_p^2) and
 *       1.75 (1-eps)/d_p, which stay finite at eps = 1.
 *   R7  Walls are half-way bounce-back: a population that would leave through a
 *       wall face returns to its node in the opposite direction after one step.
 *   R8  nu = cs^2 (tau - 1/2) dt, p = cs^2 rho (stated after Eq. VNS2), dt = 1.
 *   R9  wall_kind 1 (the paper's validation runs, Sec. "Examples and
 *       discussions", apply the non-equilibrium extrapolation scheme of Guo,
 *       Zheng & Shi 2002 at both plates): the rows y = 0 and y = ny-1 are nodes
 *       on the plates (H = ny - 1).  A plate node x_b takes
 *         f_i(x_b) = f_i^eq(eps(x_b), rho(x_f), u_b)
 *                    + [f_i(x_f) - f_i^eq(eps(x_f), rho(x_f), u(x_f))]
 *       from its fluid neighbour x_f = x_b +- e_y (rho, u by Eqs. 0moment and
 *       1moment), u_b = 0 on the lower plate and u_wall on the upper one, and
 *       relaxes towards f^eq(eps(x_b), rho_b, u_b) with no source term (the
 *       plate velocity is imposed, the drag acts on the fluid).  The paper does
 *       not say how the forcing terms meet the boundary nodes; this is the
 *       reading.  Only the y walls take this scheme (no z walls).
 *
 * Layout: f[i*N + n], n = (z*ny + y)*nx + x, N = nx*ny*nz.  eps is double[N].
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int q;              /* 9 (D2Q9) or 19 (D3Q19)                                  */
    int nx, ny, nz;     /* nz = 1 for D2Q9                                         */
    int wall_mask;      /* bit0 x, bit1 y, bit2 z: 1 = bounce-back walls, 0 = periodic */
    double tau;         /* relaxation time                                         */
    double g[3];        /* body force per unit mass (R4)                          */
    int drag_mode;      /* 0 none, 1 Darcy only, 2 Darcy + Forchheimer             */
    int k_mode;         /* 0 Ergun K(eps,d_p), F_eps(eps); 1 fixed K, F_eps;
                           2 fixed K, F_eps(eps) from the paper's formula          */
    double d_p, K, F_eps;
    double u_wall[3];   /* velocity of the upper y wall                            */
    int wall_kind;      /* y walls: 0 half-way bounce-back (R7), 1 non-equilibrium
                           extrapolation at nodes on the plates (R9)               */
} or_params;

static const double CS2 = 1.0 / 3.0;

/* R1: D2Q9 velocity set and weights (Qian et al. 1992). */
static const int D2Q9_E[9][3] = {
    {0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0},
    {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
static const double D2Q9_W[9] = {
    4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
    1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

/* R1: D3Q19 velocity set and weights. */
static const int D3Q19_E[19][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static const double D3Q19_W[19] = {
    1.0 / 3,
    1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18,
    1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36,
    1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

typedef struct {
    int q;
    int dim;
    int e[19][3];
    double w[19];
    int opp[19];
} lattice_t;

static int make_lattice(int q, lattice_t *L)
{
    const int(*E)[3];
    const double *W;
    if (q == 9) {
        E = D2Q9_E; W = D2Q9_W; L->dim = 2;
    } else if (q == 19) {
        E = D3Q19_E; W = D3Q19_W; L->dim = 3;
    } else {
        return -1;
    }
    L->q = q;
    for (int i = 0; i < q; ++i) {
        for (int a = 0; a < 3; ++a) L->e[i][a] = E[i][a];
        L->w[i] = W[i];
    }
    /* opposite direction: the one with e_j = -e_i */
    for (int i = 0; i < q; ++i) {
        L->opp[i] = -1;
        for (int j = 0; j < q; ++j)
            if (E[j][0] == -E[i][0] && E[j][1] == -E[i][1] && E[j][2] == -E[i][2])
                L->opp[i] = j;
    }
    return 0;
}

/* Exported: the velocity set, weights and opposite table (for the table pins). */
int or_lattice(int q, int *e_out, double *w_out, int *opp_out)
{
    lattice_t L;
    if (make_lattice(q, &L)) return -1;
    for (int i = 0; i < q; ++i) {
        for (int a = 0; a < 3; ++a) e_out[3 * i + a] = L.e[i][a];
        w_out[i] = L.w[i];
        opp_out[i] = L.opp[i];
    }
    return 0;
}

static int check_params(const or_params *p, lattice_t *L)
{
    if (make_lattice(p->q, L)) return -1;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return -1;
    if (p->q == 9 && p->nz != 1) return -1;
    if (!(p->tau > 0.5)) return -1;
    if (p->wall_kind != 0 && p->wall_kind != 1) return -1;
    if (p->wall_kind == 1 && (!(p->wall_mask & 2) || (p->wall_mask & 5) || p->ny < 3)) return -1;
    return 0;
}

/* R9: is row y a plate node? */
static inline int plate_row(const or_params *p, int y)
{
    return p->wall_kind == 1 && (y == 0 || y == p->ny - 1);
}

static double nu_of(const or_params *p) { return CS2 * (p->tau - 0.5); } /* R8 */

/* Drag coefficients alpha = eps^2 nu / K and beta = eps^3 F_eps / sqrt(K), with
 * the permeability K and the geometric function F_eps chosen by k_mode:
 *   k_mode 0: K = eps^3 d_p^2 / (150 (1-eps)^2) and F_eps = 1.75 / sqrt(150 eps^3)
 *             (Ergun, as quoted from Vafai), substituted in closed form (R6);
 *   k_mode 1: K and F_eps given;
 *   k_mode 2: K given, F_eps = 1.75 / sqrt(150 eps^3).
 * The derivatives d alpha/d eps and d beta/d eps are returned for the adjoint. */
static void drag_coeffs(const or_params *p, double eps, double *alpha, double *beta,
                        double *dalpha, double *dbeta)
{
    const double nu = nu_of(p);
    double a = 0, b = 0, da = 0, db = 0;
    if (p->k_mode == 0) {
        const double c = 150.0 * nu / (p->d_p * p->d_p);
        a = c * (1 - eps) * (1 - eps) / eps;
        da = -c * (1 - eps) * (1 + eps) / (eps * eps);
        b = 1.75 * (1 - eps) / p->d_p;
        db = -1.75 / p->d_p;
    } else if (p->k_mode == 1) {
        a = eps * eps * nu / p->K;
        da = 2 * eps * nu / p->K;
        b = eps * eps * eps * p->F_eps / sqrt(p->K);
        db = 3 * eps * eps * p->F_eps / sqrt(p->K);
    } else {
        const double Feps = 1.75 / sqrt(150.0 * eps * eps * eps);
        a = eps * eps * nu / p->K;
        da = 2 * eps * nu / p->K;
        b = eps * eps * eps * Feps / sqrt(p->K);     /* = 1.75 eps^1.5 / sqrt(150 K) */
        db = 1.5 * b / eps;
    }
    if (p->drag_mode == 0) { a = b = da = db = 0; }
    if (p->drag_mode == 1) { b = db = 0; }
    *alpha = a; *beta = b;
    if (dalpha) *dalpha = da;
    if (dbeta) *dbeta = db;
}

int or_drag_coeffs(const or_params *p, double eps, double *alpha, double *beta)
{
    drag_coeffs(p, eps, alpha, beta, NULL, NULL);
    return 0;
}

/* R3: the exact solution of (eps rho + alpha/2 + beta/2 |u|) u = m. */
static void velocity_solve(double R, const double m[3], double alpha, double beta, double u[3])
{
    const double a = R + 0.5 * alpha;
    const double b = 0.5 * beta;
    const double mm = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
    const double D = a + sqrt(a * a + 4.0 * b * mm);
    for (int k = 0; k < 3; ++k) u[k] = 2.0 * m[k] / D;
}

void or_velocity(double R, const double *m, double alpha, double beta, double *u)
{
    velocity_solve(R, m, alpha, beta, u);
}

/* Eq. d2q9eq for all i. */
static void equilibrium(const lattice_t *L, double eps, double rho, const double u[3], double *feq)
{
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < L->q; ++i) {
        const double eu = L->e[i][0] * u[0] + L->e[i][1] * u[1] + L->e[i][2] * u[2];
        feq[i] = L->w[i] * eps * rho *
                 (1.0 + eu / CS2 + eu * eu / (2 * CS2 * CS2) - uu / (2 * CS2));
    }
}

int or_feq(int q, double eps, double rho, const double *u, double *feq)
{
    lattice_t L;
    if (make_lattice(q, &L)) return -1;
    equilibrium(&L, eps, rho, u, feq);
    return 0;
}

/* Eq. pi / Eq. Fi: (1 - 1/(2 tau)) w_i [(e_i - u)/cs^2 + (e_i.u) e_i / cs^4] . V.
 * With V = p grad eps this is P_i, with V = F it is F_i. */
static void source_term(const lattice_t *L, double tau, const double u[3], const double V[3], double *S)
{
    const double c = 1.0 - 1.0 / (2.0 * tau);
    for (int i = 0; i < L->q; ++i) {
        const double eu = L->e[i][0] * u[0] + L->e[i][1] * u[1] + L->e[i][2] * u[2];
        double s = 0;
        for (int k = 0; k < 3; ++k)
            s += ((L->e[i][k] - u[k]) / CS2 + eu * L->e[i][k] / (CS2 * CS2)) * V[k];
        S[i] = c * L->w[i] * s;
    }
}

int or_source(int q, double tau, const double *u, const double *V, double *S)
{
    lattice_t L;
    if (make_lattice(q, &L)) return -1;
    source_term(&L, tau, u, V, S);
    return 0;
}

/* neighbour index along one axis; returns -1 when the neighbour lies past a wall */
static inline int nb(int c, int d, int n, int wall)
{
    int t = c + d;
    if (t < 0 || t >= n) {
        if (wall) return -1;
        t = (t + n) % n;
    }
    return t;
}

/* R5: grad eps(x) = (1/cs^2) sum_i w_i e_i eps~(x+e_i). */
static void grad_eps_field(const or_params *p, const lattice_t *L, const double *eps, double *grad)
{
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const long N = (long)nx * ny * nz;
    const int wx = p->wall_mask & 1, wy = (p->wall_mask >> 1) & 1, wz = (p->wall_mask >> 2) & 1;
#pragma omp parallel for collapse(2) schedule(static) if ((long)nx * ny * nz > 8192)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const long n = ((long)z * ny + y) * nx + x;
                double G[3] = {0, 0, 0};
                for (int i = 0; i < L->q; ++i) {
                    const int xs = nb(x, L->e[i][0], nx, wx);
                    const int ys = nb(y, L->e[i][1], ny, wy);
                    const int zs = nb(z, L->e[i][2], nz, wz);
                    double en;
                    if (xs < 0 || ys < 0 || zs < 0) en = eps[n];
                    else en = eps[((long)zs * ny + ys) * nx + xs];
                    for (int k = 0; k < 3; ++k) G[k] += L->w[i] * L->e[i][k] * en;
                }
                for (int k = 0; k < 3; ++k) grad[k * N + n] = G[k] / CS2;
            }
}

int or_grad_eps(const or_params *p, const double *eps, double *grad)
{
    lattice_t L;
    if (check_params(p, &L)) return -1;
    grad_eps_field(p, &L, eps, grad);
    return 0;
}

/* Macroscopic quantities of one cell from its populations f_i (pre-collision). */
typedef struct {
    double R;        /* eps*rho, Eq. 0moment */
    double rho;
    double j[3];     /* sum_i e_i f_i */
    double Pc[3];    /* p grad eps = cs^2 rho grad eps */
    double m[3];     /* right-hand side of Eq. 1moment without the drag */
    double alpha, beta, dalpha, dbeta;
    double a, b, mm, s, D;
    double u[3], un; /* velocity and its norm */
    double F[3];     /* total force: body force plus drag */
    double V[3];     /* p grad eps + F, the vector the sources act on */
} cell_t;

/* Body force per unit mass along axis k; a D2Q9 lattice has no z component. */
static inline double gcomp(const or_params *p, const lattice_t *L, int k)
{
    return k < L->dim ? p->g[k] : 0.0;
}

static void cell_moments(const or_params *p, const lattice_t *L, const double *fc, double eps,
                         const double gradc[3], cell_t *c)
{
    c->R = 0;
    for (int k = 0; k < 3; ++k) c->j[k] = 0;
    for (int i = 0; i < L->q; ++i) {
        c->R += fc[i];
        for (int k = 0; k < 3; ++k) c->j[k] += L->e[i][k] * fc[i];
    }
    c->rho = c->R / eps;
    drag_coeffs(p, eps, &c->alpha, &c->beta, &c->dalpha, &c->dbeta);
    for (int k = 0; k < 3; ++k) {
        c->Pc[k] = CS2 * c->rho * gradc[k];
        c->m[k] = c->j[k] + 0.5 * c->Pc[k] + 0.5 * c->R * gcomp(p, L, k);
    }
    c->a = c->R + 0.5 * c->alpha;
    c->b = 0.5 * c->beta;
    c->mm = sqrt(c->m[0] * c->m[0] + c->m[1] * c->m[1] + c->m[2] * c->m[2]);
    c->s = sqrt(c->a * c->a + 4.0 * c->b * c->mm);
    c->D = c->a + c->s;
    velocity_solve(c->R, c->m, c->alpha, c->beta, c->u);
    c->un = sqrt(c->u[0] * c->u[0] + c->u[1] * c->u[1] + c->u[2] * c->u[2]);
    for (int k = 0; k < 3; ++k) {
        c->F[k] = c->R * gcomp(p, L, k) - c->alpha * c->u[k] - c->beta * c->un * c->u[k];
        c->V[k] = c->Pc[k] + c->F[k];
    }
}

static void gather_cell(const lattice_t *L, const double *f, long N, long n, double *fc)
{
    for (int i = 0; i < L->q; ++i) fc[i] = f[i * N + n];
}

/* R9: populations of the plate nodes from their fluid neighbours. */
static void plate_nodes(const or_params *p, const lattice_t *L, const double *eps,
                        const double *grad, double *f)
{
    if (p->wall_kind != 1) return;
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const long N = (long)nx * ny * nz;
    for (int z = 0; z < nz; ++z)
        for (int side = 0; side < 2; ++side) {
            const int yb = side ? ny - 1 : 0, yf = side ? ny - 2 : 1;
            const double zero[3] = {0, 0, 0};
            const double *ub = side ? p->u_wall : zero;
            for (int x = 0; x < nx; ++x) {
                const long nb_ = ((long)z * ny + yb) * nx + x, nf = ((long)z * ny + yf) * nx + x;
                double fc[19], feqf[19], feqb[19], gc[3] = {grad[nf], grad[N + nf], grad[2 * N + nf]};
                cell_t c;
                gather_cell(L, f, N, nf, fc);
                cell_moments(p, L, fc, eps[nf], gc, &c);
                equilibrium(L, eps[nf], c.rho, c.u, feqf);
                equilibrium(L, eps[nb_], c.rho, ub, feqb);
                for (int i = 0; i < L->q; ++i) f[i * N + nb_] = feqb[i] + (fc[i] - feqf[i]);
            }
        }
}

/* Initial state of the validation runs: rho = 1, u = 0, so f_i = w_i eps (and
 * the plate nodes from their neighbours under R9). */
int or_init(const or_params *p, const double *eps, double *f)
{
    lattice_t L;
    if (check_params(p, &L)) return -1;
    const long N = (long)p->nx * p->ny * p->nz;
    for (int i = 0; i < L.q; ++i)
        for (long n = 0; n < N; ++n) f[i * N + n] = L.w[i] * eps[n];
    if (p->wall_kind == 1) {
        double *grad = (double *)malloc(sizeof(double) * 3 * N);
        if (!grad) return -2;
        grad_eps_field(p, &L, eps, grad);
        plate_nodes(p, &L, eps, grad, f);
        free(grad);
    }
    return 0;
}

/* rho and u of every cell from the state f (Eqs. 0moment and 1moment). */
int or_moments(const or_params *p, const double *eps, const double *f, double *rho, double *u)
{
    lattice_t L;
    if (check_params(p, &L)) return -1;
    const long N = (long)p->nx * p->ny * p->nz;
    double *grad = (double *)malloc(sizeof(double) * 3 * N);
    if (!grad) return -2;
    grad_eps_field(p, &L, eps, grad);
#pragma omp parallel for schedule(static) if (N > 8192)
    for (long n = 0; n < N; ++n) {
        double fc[19], gc[3] = {grad[n], grad[N + n], grad[2 * N + n]};
        cell_t c;
        gather_cell(&L, f, N, n, fc);
        cell_moments(p, &L, fc, eps[n], gc, &c);
        rho[n] = c.rho;
        for (int k = 0; k < L.dim; ++k) u[k * N + n] = c.u[k];
    }
    free(grad);
    return 0;
}

/* Collision in place: f (pre-collision f_i(x,t)) -> f* (post-collision). */
static void collide(const or_params *p, const lattice_t *L, const double *eps, const double *grad,
                    double *f)
{
    const long N = (long)p->nx * p->ny * p->nz;
    const double tau = p->tau;
#pragma omp parallel for schedule(static) if (N > 8192)
    for (long n = 0; n < N; ++n) {
        double fc[19], feq[19], S[19], gc[3] = {grad[n], grad[N + n], grad[2 * N + n]};
        cell_t c;
        gather_cell(L, f, N, n, fc);
        const int y = (int)((n / p->nx) % p->ny);
        if (plate_row(p, y)) {
            /* R9: relax towards the plate's equilibrium, no source term */
            const double zero[3] = {0, 0, 0};
            double R = 0;
            for (int i = 0; i < L->q; ++i) R += fc[i];
            equilibrium(L, eps[n], R / eps[n], y == 0 ? zero : p->u_wall, feq);
            for (int i = 0; i < L->q; ++i) f[i * N + n] = fc[i] - (fc[i] - feq[i]) / tau;
            continue;
        }
        cell_moments(p, L, fc, eps[n], gc, &c);
        equilibrium(L, eps[n], c.rho, c.u, feq);
        source_term(L, tau, c.u, c.V, S);   /* P_i + F_i in one call: V = p grad eps + F */
        for (int i = 0; i < L->q; ++i)
            f[i * N + n] = fc[i] - (fc[i] - feq[i]) / tau + S[i];
    }
}

/* Streaming (push): f_i(x + e_i, t+1) = f*_i(x).  Past a wall the population
 * comes back to x in the opposite direction (R7).  A moving upper y wall adds
 * 2 w_i eps rho_w (e_i . u_w)/cs^2 to the reflected population (moving-wall
 * bounce-back with the eps-weighted equilibrium; rho_w = 1). */
static void stream(const or_params *p, const lattice_t *L, const double *eps, const double *fs,
                   double *fn)
{
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const long N = (long)nx * ny * nz;
    const int wx = p->wall_mask & 1, wy = (p->wall_mask >> 1) & 1, wz = (p->wall_mask >> 2) & 1;
#pragma omp parallel for collapse(2) schedule(static) if ((long)nx * ny * nz > 8192)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const long n = ((long)z * ny + y) * nx + x;
                for (int i = 0; i < L->q; ++i) {
                    const int xd = nb(x, L->e[i][0], nx, wx);
                    const int yd = nb(y, L->e[i][1], ny, wy);
                    const int zd = nb(z, L->e[i][2], nz, wz);
                    if (xd < 0 || yd < 0 || zd < 0) {
                        double add = 0;
                        if (p->wall_kind == 0 && yd < 0 && L->e[i][1] > 0 && xd >= 0 && zd >= 0) {
                            const double eu = L->e[i][0] * p->u_wall[0] + L->e[i][1] * p->u_wall[1] +
                                              L->e[i][2] * p->u_wall[2];
                            add = 2.0 * L->w[i] * eps[n] * eu / CS2;
                        }
                        /* the reflected population carries -e_i: it is f_opp(i) at x */
                        fn[L->opp[i] * N + n] = fs[i * N + n] - add;
                    } else {
                        fn[i * N + ((long)zd * ny + yd) * nx + xd] = fs[i * N + n];
                    }
                }
            }
}

int or_stream(const or_params *p, const double *eps, const double *fs, double *fn)
{
    lattice_t L;
    if (check_params(p, &L)) return -1;
    stream(p, &L, eps, fs, fn);
    return 0;
}

int or_collide(const or_params *p, const double *eps, double *f)
{
    lattice_t L;
    if (check_params(p, &L)) return -1;
    const long N = (long)p->nx * p->ny * p->nz;
    double *grad = (double *)malloc(sizeof(double) * 3 * N);
    if (!grad) return -2;
    grad_eps_field(p, &L, eps, grad);
    collide(p, &L, eps, grad, f);
    free(grad);
    return 0;
}

/* nsteps of the final LBE: collide, then stream.  f holds f(x,t) on entry and
 * f(x,t+nsteps) on return. */
int or_run(const or_params *p, const double *eps, double *f, int nsteps)
{
    lattice_t L;
    if (check_params(p, &L)) return -1;
    const long N = (long)p->nx * p->ny * p->nz;
    double *grad = (double *)malloc(sizeof(double) * 3 * N);
    double *tmp = (double *)malloc(sizeof(double) * L.q * N);
    if (!grad || !tmp) { free(grad); free(tmp); return -2; }
    grad_eps_field(p, &L, eps, grad);
    for (int t = 0; t < nsteps; ++t) {
        plate_nodes(p, &L, eps, grad, f);     /* R9 (no-op for bounce-back walls) */
        collide(p, &L, eps, grad, f);
        stream(p, &L, eps, f, tmp);
        memcpy(f, tmp, sizeof(double) * L.q * N);
    }
    plate_nodes(p, &L, eps, grad, f);
    free(grad);
    free(tmp);
    return 0;
}

/* Outlet flux J = sum over the plane x = x_out of eps*rho*u_x (Eq. 1moment). */
int or_flux(const or_params *p, const double *eps, const double *f, int x_out, double *J)
{
    lattice_t L;
    if (check_params(p, &L)) return -1;
    if (x_out < 0 || x_out >= p->nx) return -1;
    const long N = (long)p->nx * p->ny * p->nz;
    double *grad = (double *)malloc(sizeof(double) * 3 * N);
    if (!grad) return -2;
    grad_eps_field(p, &L, eps, grad);
    double s = 0;
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y) {
            const long n = ((long)z * p->ny + y) * p->nx + x_out;
            double fc[19], gc[3] = {grad[n], grad[N + n], grad[2 * N + n]};
            cell_t c;
            gather_cell(&L, f, N, n, fc);
            cell_moments(p, &L, fc, eps[n], gc, &c);
            s += c.R * c.u[0];
        }
    free(grad);
    *J = s;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Discrete adjoint of the run above (reverse mode, hand-derived, FP64).      */
/*                                                                            */
/* With f(t+1) = Stream(Collide(f(t); eps)), f(0) = w eps and J = flux(f(T)),  */
/*   dJ/deps = d flux/d eps |_f  +  sum_t (d Collide_t / d eps |_f)^T mu_t     */
/*           + sum_i w_i lambda_i(0),                                         */
/* where lambda(t) = dJ/df(t) and mu_t = Stream^T lambda(t+1) = dJ/df*(t).      */
/* eps enters each cell through eps(x) (rho = eps rho / eps, alpha, beta) and  */
/* through grad eps; the latter is collected per cell and mapped back through  */
/* the transposed stencil of R5 at the end.                                    */
/* ------------------------------------------------------------------------- */

/* Reverse of cell_moments: given the adjoints of u, F-independent outputs R and V
 * (Rbar, ubar, Vbar), add the adjoint of every f_i into fbar and return the
 * adjoints of eps(x) and grad eps(x). */
static void cell_moments_vjp(const or_params *p, const lattice_t *L, const cell_t *c, double eps,
                             const double gradc[3], double Rbar, double ubar[3], const double Vbar[3],
                             double *fbar, double *epsbar, double gbar[3])
{
    double Pcbar[3], Fbar[3], mbar[3], jbar[3];
    double alphabar = 0, betabar = 0;
    /* V = Pc + F */
    for (int k = 0; k < 3; ++k) { Pcbar[k] = Vbar[k]; Fbar[k] = Vbar[k]; }
    /* F = R g - alpha u - beta |u| u */
    double Fu = 0;
    for (int k = 0; k < 3; ++k) {
        Rbar += Fbar[k] * gcomp(p, L, k);
        Fu += Fbar[k] * c->u[k];
    }
    alphabar += -Fu;
    betabar += -c->un * Fu;
    for (int k = 0; k < 3; ++k) {
        ubar[k] += -c->alpha * Fbar[k] - c->beta * c->un * Fbar[k];
        if (c->un > 0) ubar[k] += -c->beta * Fu * c->u[k] / c->un;
    }
    /* u = 2 m / D, D = a + s, s = sqrt(a^2 + 4 b |m|) */
    double ubar_u = 0;
    for (int k = 0; k < 3; ++k) {
        mbar[k] = 2.0 * ubar[k] / c->D;
        ubar_u += ubar[k] * c->u[k];
    }
    const double Dbar = -ubar_u / c->D;
    double abar = Dbar, sbar = Dbar;
    abar += sbar * c->a / c->s;
    const double bbar = sbar * 2.0 * c->mm / c->s;
    const double mmbar = sbar * 2.0 * c->b / c->s;
    if (c->mm > 0)
        for (int k = 0; k < 3; ++k) mbar[k] += mmbar * c->m[k] / c->mm;
    /* a = R + alpha/2, b = beta/2 */
    Rbar += abar;
    alphabar += 0.5 * abar;
    betabar += 0.5 * bbar;
    /* m = j + Pc/2 + R g/2 */
    for (int k = 0; k < 3; ++k) {
        jbar[k] = mbar[k];
        Pcbar[k] += 0.5 * mbar[k];
        Rbar += 0.5 * mbar[k] * gcomp(p, L, k);
    }
    /* Pc = cs^2 rho grad eps */
    double rhobar = 0;
    for (int k = 0; k < 3; ++k) {
        rhobar += CS2 * Pcbar[k] * gradc[k];
        gbar[k] += CS2 * c->rho * Pcbar[k];
    }
    /* rho = R / eps */
    Rbar += rhobar / eps;
    *epsbar += -rhobar * c->R / (eps * eps);
    /* alpha(eps), beta(eps) */
    *epsbar += alphabar * c->dalpha + betabar * c->dbeta;
    /* R = sum f, j = sum e f */
    for (int i = 0; i < L->q; ++i)
        fbar[i] += Rbar + L->e[i][0] * jbar[0] + L->e[i][1] * jbar[1] + L->e[i][2] * jbar[2];
}

/* Reverse of the collision of one cell: mu = dJ/df*, returns lambda = dJ/df in lam. */
static void collide_vjp(const or_params *p, const lattice_t *L, const double *fc, double eps,
                        const double gradc[3], const double *mu, double *lam, double *epsbar,
                        double gbar[3])
{
    cell_t c;
    cell_moments(p, L, fc, eps, gradc, &c);
    const double tau = p->tau;
    const double ct = 1.0 - 1.0 / (2.0 * tau);
    const double uu = c.u[0] * c.u[0] + c.u[1] * c.u[1] + c.u[2] * c.u[2];
    double Rbar = 0, ubar[3] = {0, 0, 0}, Vbar[3] = {0, 0, 0};
    for (int i = 0; i < L->q; ++i) {
        /* f*_i = f_i - (f_i - feq_i)/tau + S_i */
        lam[i] = (1.0 - 1.0 / tau) * mu[i];
        const double feqbar = mu[i] / tau;
        const double Sbar = mu[i];
        const double eu = L->e[i][0] * c.u[0] + L->e[i][1] * c.u[1] + L->e[i][2] * c.u[2];
        /* feq_i = w_i R (1 + eu/cs2 + eu^2/(2cs4) - uu/(2cs2)), R = eps rho */
        Rbar += feqbar * L->w[i] * (1.0 + eu / CS2 + eu * eu / (2 * CS2 * CS2) - uu / (2 * CS2));
        /* S_i = ct w_i [(e_i - u)/cs2 + eu e_i/cs4] . V */
        double eV = 0;
        for (int k = 0; k < 3; ++k) eV += L->e[i][k] * c.V[k];
        for (int k = 0; k < 3; ++k) {
            ubar[k] += feqbar * L->w[i] * c.R *
                       (L->e[i][k] / CS2 + eu * L->e[i][k] / (CS2 * CS2) - c.u[k] / CS2);
            Vbar[k] += Sbar * ct * L->w[i] * ((L->e[i][k] - c.u[k]) / CS2 + eu * L->e[i][k] / (CS2 * CS2));
            ubar[k] += Sbar * ct * L->w[i] * (-c.V[k] / CS2 + eV * L->e[i][k] / (CS2 * CS2));
        }
    }
    cell_moments_vjp(p, L, &c, eps, gradc, Rbar, ubar, Vbar, lam, epsbar, gbar);
}

/* Transposed R5 stencil: adds to epsbar the contribution of gbar (dJ/d grad eps). */
static void grad_eps_transpose(const or_params *p, const lattice_t *L, const double *gbar,
                               double *epsbar)
{
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const long N = (long)nx * ny * nz;
    const int wx = p->wall_mask & 1, wy = (p->wall_mask >> 1) & 1, wz = (p->wall_mask >> 2) & 1;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const long n = ((long)z * ny + y) * nx + x;
                for (int i = 0; i < L->q; ++i) {
                    const int xs = nb(x, L->e[i][0], nx, wx);
                    const int ys = nb(y, L->e[i][1], ny, wy);
                    const int zs = nb(z, L->e[i][2], nz, wz);
                    const long t = (xs < 0 || ys < 0 || zs < 0) ? n : ((long)zs * ny + ys) * nx + xs;
                    double s = 0;
                    for (int k = 0; k < 3; ++k) s += L->w[i] * L->e[i][k] * gbar[k * N + n];
                    epsbar[t] += s / CS2;
                }
            }
}

/* Transposed streaming: mu = Stream^T lam (mu = dJ/df*, lam = dJ/df(t+1)). */
static void stream_transpose(const or_params *p, const lattice_t *L, const double *lam, double *mu,
                             double *epsbar)
{
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const long N = (long)nx * ny * nz;
    const int wx = p->wall_mask & 1, wy = (p->wall_mask >> 1) & 1, wz = (p->wall_mask >> 2) & 1;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const long n = ((long)z * ny + y) * nx + x;
                for (int i = 0; i < L->q; ++i) {
                    const int xd = nb(x, L->e[i][0], nx, wx);
                    const int yd = nb(y, L->e[i][1], ny, wy);
                    const int zd = nb(z, L->e[i][2], nz, wz);
                    if (xd < 0 || yd < 0 || zd < 0) {
                        const double lb = lam[L->opp[i] * N + n];
                        mu[i * N + n] = lb;
                        /* moving-wall term -2 w_i eps (e_i.u_w)/cs2 depends on eps(x) */
                        if (p->wall_kind == 0 && yd < 0 && L->e[i][1] > 0 && xd >= 0 && zd >= 0) {
                            const double eu = L->e[i][0] * p->u_wall[0] + L->e[i][1] * p->u_wall[1] +
                                              L->e[i][2] * p->u_wall[2];
                            epsbar[n] += -2.0 * L->w[i] * eu / CS2 * lb;
                        }
                    } else {
                        mu[i * N + n] = lam[i * N + ((long)zd * ny + yd) * nx + xd];
                    }
                }
            }
}

/* dJ/deps for J = flux(f(T)) after nsteps from f(0) = w eps.  Stores the whole
 * trajectory (small problems only).  Returns J as well. */
int or_adjoint(const or_params *p, const double *eps, int nsteps, int x_out, double *dJdeps,
               double *J_out)
{
    lattice_t L;
    if (check_params(p, &L)) return -1;
    if (x_out < 0 || x_out >= p->nx || nsteps < 0) return -1;
    if (p->wall_kind != 0) return -1;    /* the adjoint covers bounce-back walls only */
    const int Q = L.q;
    const long N = (long)p->nx * p->ny * p->nz;
    double *traj = (double *)malloc(sizeof(double) * Q * N * ((long)nsteps + 1));
    double *grad = (double *)malloc(sizeof(double) * 3 * N);
    double *gbar = (double *)calloc(3 * N, sizeof(double));
    double *lam = (double *)calloc(Q * N, sizeof(double));
    double *mu = (double *)malloc(sizeof(double) * Q * N);
    if (!traj || !grad || !gbar || !lam || !mu) {
        free(traj); free(grad); free(gbar); free(lam); free(mu);
        return -2;
    }
    grad_eps_field(p, &L, eps, grad);
    /* forward, keeping f(t) for t = 0..T */
    double *f0 = traj;
    for (int i = 0; i < Q; ++i)
        for (long n = 0; n < N; ++n) f0[i * N + n] = L.w[i] * eps[n];
    for (int t = 0; t < nsteps; ++t) {
        double *ft = traj + (long)t * Q * N, *fn = traj + (long)(t + 1) * Q * N;
        memcpy(mu, ft, sizeof(double) * Q * N);
        collide(p, &L, eps, grad, mu);
        stream(p, &L, eps, mu, fn);
    }
    const double *fT = traj + (long)nsteps * Q * N;
    for (long n = 0; n < N; ++n) dJdeps[n] = 0;
    /* seed: J = sum_{x = x_out} R u_x, i.e. Rbar = u_x, ubar = (R, 0, 0) */
    double J = 0;
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y) {
            const long n = ((long)z * p->ny + y) * p->nx + x_out;
            double fc[19], gc[3] = {grad[n], grad[N + n], grad[2 * N + n]};
            double fb[19] = {0}, Vbar[3] = {0, 0, 0}, g3[3] = {0, 0, 0};
            cell_t c;
            gather_cell(&L, fT, N, n, fc);
            cell_moments(p, &L, fc, eps[n], gc, &c);
            J += c.R * c.u[0];
            double ubar[3] = {c.R, 0, 0};
            cell_moments_vjp(p, &L, &c, eps[n], gc, c.u[0], ubar, Vbar, fb, &dJdeps[n], g3);
            for (int i = 0; i < Q; ++i) lam[i * N + n] = fb[i];
            for (int k = 0; k < 3; ++k) gbar[k * N + n] += g3[k];
        }
    /* backward through the steps */
    for (int t = nsteps - 1; t >= 0; --t) {
        const double *ft = traj + (long)t * Q * N;
        stream_transpose(p, &L, lam, mu, dJdeps);
        for (long n = 0; n < N; ++n) {
            double fc[19], mc[19], lc[19], gc[3] = {grad[n], grad[N + n], grad[2 * N + n]};
            double g3[3] = {0, 0, 0};
            gather_cell(&L, ft, N, n, fc);
            gather_cell(&L, mu, N, n, mc);
            collide_vjp(p, &L, fc, eps[n], gc, mc, lc, &dJdeps[n], g3);
            for (int i = 0; i < Q; ++i) lam[i * N + n] = lc[i];
            for (int k = 0; k < 3; ++k) gbar[k * N + n] += g3[k];
        }
    }
    /* f(0) = w eps */
    for (long n = 0; n < N; ++n)
        for (int i = 0; i < Q; ++i) dJdeps[n] += L.w[i] * lam[i * N + n];
    grad_eps_transpose(p, &L, gbar, dJdeps);
    if (J_out) *J_out = J;
    free(traj); free(grad); free(gbar); free(lam); free(mu);
    return 0;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
