/*
 * Plain FP64 CPU oracle for the free-energy binary-fluid lattice Boltzmann
 * step of Pooley, Kusumaatmaja & Yeomans, "Contact line dynamics in binary
 * lattice Boltzmann simulations" (arXiv:0812.1282).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library may link, load or
 * call this file; only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code with the CUDA path.
 *
 * The code is deliberately literal and slow: one pass per algorithmic step
 * over the whole lattice, the equilibria written with the generic
 * e_ia e_ib sums of the Appendix, and the MRT collision as the dense
 * 9x9 products M^-1 S M of Sec. III.B.  All arithmetic is double precision.
 *
 * Lattice conventions (Sec. III.A): velocities in the paper's order
 *   e0=(0,0) e1=(1,0) e2=(-1,0) e3=(0,1) e4=(0,-1)
 *   e5=(1,1) e6=(-1,-1) e7=(-1,1) e8=(1,-1),   c = dx = dt = 1.
 * Arrays are [population][y][x] with x fastest, nx columns, ny rows.
 * x is always periodic.  y is periodic (walls == 0) or bounded by mid-link
 * bounce-back walls below row 0 and above row ny-1 (walls == 1).
 *
 * The stored state is the post-collision population set f'(t), g'(t).
 * One call of orc_step advances it by: pull-stream (Eqs. stream1-2, with
 * bounce-back), moments (Step 1, Eq. moments), derivatives (Eq. best with the
 * wetting ghost rows), chemical potential / pressure (Eqs. chempot, p0),
 * Step 2 (zero equilibrium velocity at boundary nodes), equilibria (Eq.
 * equilibrium, feq0) and BGK (Eqs. latbolt, gevo) or MRT (Eqs. mrtlb, Matrix,
 * diag) collision.
 *
 * Readings of points the paper leaves open (kept identical on the CUDA side
 * by independent code):
 *  - wetting gradient h is the inward-normal derivative of phi at a wall
 *    (xi = kappa*h, Sec. II); a ghost row mirrors phi about the boundary row:
 *    phi(x,-1) = phi(x,1) - 2 h_bottom, phi(x,ny) = phi(x,ny-2) - 2 h_top,
 *    which makes the isotropic y-derivative at the boundary row equal to the
 *    imposed inward gradient exactly (with wetting_rule = 1 instead the
 *    one-sided difference across the wall plane: phi(x,-1) = phi(x,0) - h);
 *  - boundary nodes of Step 2 are the fluid rows adjacent to a wall;
 *  - conserved-moment rates are the literal zeros of Eq. diag (optionally,
 *    step2_relax_momentum: rate 1 for the momentum rows on Step-2 nodes).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct orc_params {
    double a, kappa;          /* psi = a(-phi^2/2 + phi^4/4), Eq. bulkfe     */
    double gamma_mob;         /* Gamma of the g equilibrium, Eq. Mobility   */
    double tau_phi;           /* g relaxation time, Eq. gevo                */
    double tau_alpha;         /* tau_rho in the phi=+1 phase, Eq. tau       */
    double tau_beta;          /* tau_rho in the phi=-1 phase, Eq. tau       */
    double h_bottom, h_top;   /* inward normal d(phi)/dn at the walls       */
    int collision;            /* 0 = BGK (Eq. latbolt), 1 = MRT (Eq. mrtlb) */
    int zero_u_at_walls;      /* Step 2 of Sec. V                           */
    int walls;                /* 1 = walls at y=0 and y=ny-1, 0 = periodic  */
    int mrt_all_rates;        /* test mode: every S entry equal to omega    */
    int step2_relax_momentum; /* MRT: momentum rows relax at rate 1 on Step-2
                                 nodes (default 0: the literal zeros of Eq. diag) */
    int mrt_lut;              /* MRT: 0 = exact tau(phi); n >= 2 = the nearest of n
                                 tabulated viscosities (Sec. V lookup table)  */
    int wetting_rule;         /* ghost of the wetting condition (Sec. II): 0 = mirror
                                 about the boundary row, phi(-1) = phi(1) - 2h; 1 =
                                 one-sided at the wall plane, phi(-1) = phi(0) - h */
} orc_params;

/* Mirror distance of the wetting ghost: 2 (about the boundary row) or 1
 * (one-sided difference across the wall plane). */
static int wet_k(const orc_params* p) { return p->wetting_rule ? 1 : 2; }

/* ---------------------------------------------------------------- lattice */
static const int EX[9] = {0, 1, -1, 0, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 0, 1, -1, 1, -1, 1, -1};
static const int OPP[9] = {0, 2, 1, 4, 3, 6, 5, 8, 7};

/* Appendix weights for i = 1..8 (index 0 unused: it follows from Eq. feq0) */
static const double WI[9] = {0.0, 1.0 / 3, 1.0 / 3, 1.0 / 3, 1.0 / 3,
                             1.0 / 12, 1.0 / 12, 1.0 / 12, 1.0 / 12};
static const double WXX[9] = {0.0, 1.0 / 3, 1.0 / 3, -1.0 / 6, -1.0 / 6,
                              -1.0 / 24, -1.0 / 24, -1.0 / 24, -1.0 / 24};
static const double WYY[9] = {0.0, -1.0 / 6, -1.0 / 6, 1.0 / 3, 1.0 / 3,
                              -1.0 / 24, -1.0 / 24, -1.0 / 24, -1.0 / 24};
static const double WXY[9] = {0.0, 0.0, 0.0, 0.0, 0.0,
                              1.0 / 4, 1.0 / 4, -1.0 / 4, -1.0 / 4};

/* Eq. Matrix, rows as printed (columns follow the velocity order above). */
static const double MM[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},
    {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},
    {0, 1, -1, 0, 0, 1, -1, -1, 1},
    {0, -2, 2, 0, 0, 1, -1, -1, 1},
    {0, 0, 0, 1, -1, 1, -1, 1, -1},
    {0, 0, 0, -2, 2, 1, -1, 1, -1},
    {0, 1, 1, -1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, 1, -1, -1},
};

/* Eq. best: isotropic first derivative (x) and Laplacian, indexed
 * [row][col] with row = dy+1 (bottom to top) and col = dx+1. */
static const double DX_STENCIL[3][3] = {
    {-1, 0, 1}, {-4, 0, 4}, {-1, 0, 1}};
static const double LAP_STENCIL[3][3] = {
    {1, 4, 1}, {4, -20, 4}, {1, 4, 1}};

static int g_threads = 0;

void orc_set_threads(int n) { g_threads = n; }

int orc_get_threads(void)
{
#ifdef _OPENMP
    return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

/* M^-1_ij = M_ji / sum_k M_jk^2 (orthogonal rows, Sec. III.B). */
static void mrt_inverse(double minv[9][9])
{
    for (int j = 0; j < 9; ++j) {
        double norm = 0.0;
        for (int k = 0; k < 9; ++k) norm += MM[j][k] * MM[j][k];
        for (int i = 0; i < 9; ++i) minv[i][j] = MM[j][i] / norm;
    }
}

void orc_mrt_matrix(double* m_out, double* minv_out)
{
    double minv[9][9];
    mrt_inverse(minv);
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j) {
            m_out[i * 9 + j] = MM[i][j];
            minv_out[i * 9 + j] = minv[i][j];
        }
}

static inline int wrap(int v, int n) { return ((v % n) + n) % n; }

/* tau_rho at a node of order parameter phi: Eq. tau, or with the lookup
 * table of Sec. V (MRT only) the nearest of mrt_lut values spaced evenly
 * between the two bulk values (ends included; beyond them the end value). */
double orc_node_tau(const orc_params* p, double phi)
{
    const double tau = p->tau_beta + 0.5 * (phi + 1.0) * (p->tau_alpha - p->tau_beta);
    if (p->collision != 1 || p->mrt_lut < 2 || p->tau_alpha == p->tau_beta) return tau;
    const double lo = p->tau_alpha < p->tau_beta ? p->tau_alpha : p->tau_beta;
    const double hi = p->tau_alpha < p->tau_beta ? p->tau_beta : p->tau_alpha;
    const double step = (hi - lo) / (p->mrt_lut - 1);
    double k = nearbyint((tau - lo) / step);
    if (k < 0.0) k = 0.0;
    if (k > p->mrt_lut - 1) k = p->mrt_lut - 1;
    return lo + k * step;
}

/* --------------------------------------------------------- equilibria */
/* Eq. equilibrium and Eq. feq0 at one node.  u is the velocity used in the
 * equilibrium (zero at Step-2 boundary nodes). */
void orc_node_equilibrium(const orc_params* p, double rho, double phi,
                          double ux, double uy, double dphix, double dphiy,
                          double lap, double* feq, double* geq)
{
    const double a = p->a, kappa = p->kappa;
    const double u[2] = {ux, uy};
    const double d[2] = {dphix, dphiy};
    /* Eq. p0 and Eq. chempot */
    const double p0 = rho / 3.0 + a * (-0.5 * phi * phi + 0.75 * phi * phi * phi * phi);
    const double mu = a * (-phi + phi * phi * phi) - kappa * lap;
    double fsum = 0.0, gsum = 0.0;
    for (int i = 1; i < 9; ++i) {
        const double e[2] = {(double)EX[i], (double)EY[i]};
        double eu = 0.0, quad = 0.0;
        for (int al = 0; al < 2; ++al) {
            eu += e[al] * u[al];
            for (int be = 0; be < 2; ++be) {
                const double delta = (al == be) ? 1.0 : 0.0;
                quad += 1.5 * (e[al] * e[be] - delta / 3.0) * u[al] * u[be];
            }
        }
        feq[i] = WI[i] * (p0 - kappa * phi * lap + rho * eu + rho * quad) +
                 kappa * (WXX[i] * d[0] * d[0] + WYY[i] * d[1] * d[1] +
                          WXY[i] * d[0] * d[1]);
        geq[i] = WI[i] * (p->gamma_mob * mu + phi * eu + phi * quad);
        fsum += feq[i];
        gsum += geq[i];
    }
    feq[0] = rho - fsum;
    geq[0] = phi - gsum;
}

/* Collision of one node's f (Eq. latbolt or Eq. mrtlb) given its
 * equilibrium, omega = 1/tau_rho and the inverse moment matrix.
 * step2_node: the node is a Step-2 boundary node (only matters for MRT
 * with step2_relax_momentum set). */
static void collide_f(const orc_params* p, const double minv[9][9], const double* f,
                      const double* feq, double omega, int step2_node, double* fout)
{
    if (p->collision == 0) {
        for (int i = 0; i < 9; ++i) fout[i] = f[i] - omega * (f[i] - feq[i]);
        return;
    }
    double s[9] = {0.0, 1.0, 1.0, 0.0, 1.0, 0.0, 1.0, omega, omega}; /* Eq. diag */
    if (step2_node && p->step2_relax_momentum) {
        s[3] = 1.0; /* alternative reading: the momentum of a Step-2 node */
        s[5] = 1.0; /* relaxes to its zero-velocity equilibrium           */
    }
    if (p->mrt_all_rates)
        for (int k = 0; k < 9; ++k) s[k] = omega;
    double m[9];
    for (int k = 0; k < 9; ++k) {
        double acc = 0.0;
        for (int j = 0; j < 9; ++j) acc += MM[k][j] * (f[j] - feq[j]);
        m[k] = s[k] * acc;
    }
    for (int i = 0; i < 9; ++i) {
        double acc = 0.0;
        for (int k = 0; k < 9; ++k) acc += minv[i][k] * m[k];
        fout[i] = f[i] - acc;
    }
}

void orc_node_collide_f(const orc_params* p, const double* f, const double* feq,
                        double omega, int step2_node, double* fout)
{
    double minv[9][9];
    mrt_inverse(minv);
    collide_f(p, minv, f, feq, omega, step2_node, fout);
}

/* ------------------------------------------------------ phi derivatives */
/* phi at (x, y) with the wetting ghost rows outside the walls. */
static double phi_at(const orc_params* p, int nx, int ny, const double* phi,
                     int x, int y)
{
    x = wrap(x, nx);
    if (!p->walls) return phi[(size_t)wrap(y, ny) * nx + x];
    const int k = wet_k(p);
    if (y < 0) return phi[(size_t)(k - 1) * nx + x] - k * p->h_bottom;
    if (y >= ny) return phi[(size_t)(ny - k) * nx + x] - k * p->h_top;
    return phi[(size_t)y * nx + x];
}

/* Eq. best applied at every node: d/dx, d/dy (the transpose of the printed
 * x stencil) and the nine-point Laplacian. */
void orc_phi_derivatives(const orc_params* p, int nx, int ny, const double* phi,
                         double* dx, double* dy, double* lap)
{
    int y;
#pragma omp parallel for num_threads(orc_get_threads()) schedule(static)
    for (y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            double sx = 0.0, sy = 0.0, sl = 0.0;
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) {
                    const double v = phi_at(p, nx, ny, phi, x + c - 1, y + r - 1);
                    sx += DX_STENCIL[r][c] * v;
                    sy += DX_STENCIL[c][r] * v;
                    sl += LAP_STENCIL[r][c] * v;
                }
            const size_t k = (size_t)y * nx + x;
            dx[k] = sx / 12.0;
            dy[k] = sy / 12.0;
            lap[k] = sl / 6.0;
        }
    }
}

/* ------------------------------------------------------- initial fields */
/* Drop of radius R centred at (cx, cy), phi=+1 inside, tanh profile of width
 * l = sqrt(2 kappa / a) (the flat-interface solution of Eq. chempot). */
void orc_phi_drop(const orc_params* p, int nx, int ny, double R, double cx,
                  double cy, double* phi)
{
    const double l = sqrt(2.0 * p->kappa / p->a);
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            const double d = sqrt((x - cx) * (x - cx) + (y - cy) * (y - cy));
            phi[(size_t)y * nx + x] = tanh((R - d) / l);
        }
}

/* SplitMix64 (Steele, Lea & Flood 2014), used as a counter-based generator:
 * draw k of a stream seeded with s is mix(s + (k+1) * golden_gamma). */
static uint64_t splitmix64_draw(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t orc_splitmix64(uint64_t seed, uint64_t k) { return splitmix64_draw(seed, k); }

/* phi uniform in [-amp, amp): node (x, y) takes draw k = y*nx + x. */
void orc_phi_random(int nx, int ny, double amp, uint64_t seed, double* phi)
{
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            const uint64_t k = (uint64_t)y * (uint64_t)nx + (uint64_t)x;
            const double u = (double)(splitmix64_draw(seed, k) >> 11) * 0x1.0p-53;
            phi[(size_t)k] = amp * (2.0 * u - 1.0);
        }
}

/* Initial populations: f = f^eq and g = g^eq of phi0 with rho = 1, u = 0
 * (the stored state is post-collision; colliding an equilibrium returns it). */
void orc_init(const orc_params* p, int nx, int ny, const double* phi0,
              double* f, double* g)
{
    const size_t n = (size_t)nx * ny;
    double* dx = malloc(n * sizeof(double));
    double* dy = malloc(n * sizeof(double));
    double* lap = malloc(n * sizeof(double));
    orc_phi_derivatives(p, nx, ny, phi0, dx, dy, lap);
    for (size_t k = 0; k < n; ++k) {
        double feq[9], geq[9];
        orc_node_equilibrium(p, 1.0, phi0[k], 0.0, 0.0, dx[k], dy[k], lap[k], feq, geq);
        for (int i = 0; i < 9; ++i) {
            f[(size_t)i * n + k] = feq[i];
            g[(size_t)i * n + k] = geq[i];
        }
    }
    free(dx);
    free(dy);
    free(lap);
}

/* --------------------------------------------------------- time step */
/* Pull-stream one population set: out_i(r) = in_i(r - e_i), or the reversed
 * own population in_opp(i)(r) when r - e_i lies in a wall (mid-link
 * bounce-back, Sec. IV.B / Fig. 4a). */
static void stream_pull(const orc_params* p, int nx, int ny, const double* in,
                        double* out)
{
    const size_t n = (size_t)nx * ny;
    int y;
#pragma omp parallel for num_threads(orc_get_threads()) schedule(static)
    for (y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x)
            for (int i = 0; i < 9; ++i) {
                const int sx = wrap(x - EX[i], nx);
                int sy = y - EY[i];
                double v;
                if (p->walls && (sy < 0 || sy >= ny)) {
                    v = in[(size_t)OPP[i] * n + (size_t)y * nx + x];
                } else {
                    sy = wrap(sy, ny);
                    v = in[(size_t)i * n + (size_t)sy * nx + sx];
                }
                out[(size_t)i * n + (size_t)y * nx + x] = v;
            }
}

static int is_boundary_node(const orc_params* p, int ny, int y)
{
    return p->walls && (y == 0 || y == ny - 1);
}

void orc_step(const orc_params* p, int nx, int ny, double* f, double* g, int nsteps)
{
    const size_t n = (size_t)nx * ny;
    double* fs = malloc(9 * n * sizeof(double));
    double* gs = malloc(9 * n * sizeof(double));
    double* rho = malloc(n * sizeof(double));
    double* phi = malloc(n * sizeof(double));
    double* ux = malloc(n * sizeof(double));
    double* uy = malloc(n * sizeof(double));
    double* dx = malloc(n * sizeof(double));
    double* dy = malloc(n * sizeof(double));
    double* lap = malloc(n * sizeof(double));

    double minv[9][9];
    mrt_inverse(minv);

    for (int s = 0; s < nsteps; ++s) {
        /* Eqs. stream1-2 (pull form) with bounce-back */
        stream_pull(p, nx, ny, f, fs);
        stream_pull(p, nx, ny, g, gs);

        /* Step 1: Eq. moments */
        long long k;
#pragma omp parallel for num_threads(orc_get_threads()) schedule(static)
        for (k = 0; k < (long long)n; ++k) {
            double r = 0.0, ph = 0.0, jx = 0.0, jy = 0.0;
            for (int i = 0; i < 9; ++i) {
                const double fi = fs[(size_t)i * n + k];
                r += fi;
                jx += fi * EX[i];
                jy += fi * EY[i];
                ph += gs[(size_t)i * n + k];
            }
            rho[k] = r;
            phi[k] = ph;
            ux[k] = jx / r;
            uy[k] = jy / r;
        }

        /* Eq. best with the wetting ghost rows */
        orc_phi_derivatives(p, nx, ny, phi, dx, dy, lap);

        /* Step 2, equilibria, Step 3 collision */
        int y;
#pragma omp parallel for num_threads(orc_get_threads()) schedule(static)
        for (y = 0; y < ny; ++y) {
            for (int x = 0; x < nx; ++x) {
                const size_t kk = (size_t)y * nx + x;
                double ueqx = ux[kk], ueqy = uy[kk];
                const int step2_node = p->zero_u_at_walls && is_boundary_node(p, ny, y);
                if (step2_node) {
                    ueqx = 0.0;
                    ueqy = 0.0;
                }
                double feq[9], geq[9], fin[9], fout[9];
                orc_node_equilibrium(p, rho[kk], phi[kk], ueqx, ueqy, dx[kk], dy[kk],
                                     lap[kk], feq, geq);
                /* Eq. tau */
                const double tau = orc_node_tau(p, phi[kk]); /* Eq. tau */
                const double omega = 1.0 / tau;
                for (int i = 0; i < 9; ++i) fin[i] = fs[(size_t)i * n + kk];
                collide_f(p, minv, fin, feq, omega, step2_node, fout);
                for (int i = 0; i < 9; ++i) {
                    f[(size_t)i * n + kk] = fout[i];
                    const double gi = gs[(size_t)i * n + kk];
                    g[(size_t)i * n + kk] = gi - (gi - geq[i]) / p->tau_phi; /* Eq. gevo */
                }
            }
        }
    }
    free(fs);
    free(gs);
    free(rho);
    free(phi);
    free(ux);
    free(uy);
    free(dx);
    free(dy);
    free(lap);
}

/* Observables of the stored (post-collision) state: Eq. moments. */
void orc_moments(int nx, int ny, const double* f, const double* g, double* rho,
                 double* phi, double* ux, double* uy)
{
    const size_t n = (size_t)nx * ny;
    for (size_t k = 0; k < n; ++k) {
        double r = 0.0, ph = 0.0, jx = 0.0, jy = 0.0;
        for (int i = 0; i < 9; ++i) {
            const double fi = f[(size_t)i * n + k];
            r += fi;
            jx += fi * EX[i];
            jy += fi * EY[i];
            ph += g[(size_t)i * n + k];
        }
        rho[k] = r;
        phi[k] = ph;
        ux[k] = jx / r;
        uy[k] = jy / r;
    }
}

/* One time step evaluated only on the nodes of the window
 * [x0, x1) x [y0, y1), reading a band of full-width rows
 * [band_y0, band_y0 + band_rows) of a larger lattice (nx, ny).  The band
 * must hold every row within two rows of the window (or reach the wall).
 * Output arrays are [9][y1-y0][x1-x0].  Used to check sampled nodes of
 * lattices too large for a full oracle run. */
int orc_step_window(const orc_params* p, int nx, int ny, int band_y0,
                    int band_rows, const double* fband, const double* gband,
                    int x0, int x1, int y0, int y1, double* fout_w, double* gout_w)
{
    if (x0 < 0 || x1 > nx || x0 >= x1 || y0 < 0 || y1 > ny || y0 >= y1) return -1;
    /* every source row of the pull must lie inside the band */
    for (int y = y0 - 2; y <= y1 + 1; ++y) {
        if (p->walls && (y < 0 || y >= ny)) continue;
        const int by = (p->walls ? y : wrap(y, ny)) - band_y0;
        if (by < 0 || by >= band_rows) return -1;
    }
    const size_t bn = (size_t)nx * band_rows;
    const int wx = x1 - x0, wy = y1 - y0;
    /* rows of the window plus a one-row ring for the stencil */
    const int ry0 = y0 - 1, ry1 = y1 + 1;
    const int rrows = ry1 - ry0;
    double* fs = malloc(9 * (size_t)nx * rrows * sizeof(double));
    double* gs = malloc(9 * (size_t)nx * rrows * sizeof(double));
    double* phi_full = malloc((size_t)nx * rrows * sizeof(double));
    const size_t rn = (size_t)nx * rrows;
    double minv[9][9];
    mrt_inverse(minv);
    /* pull-stream the rows of interest */
    for (int y = ry0; y < ry1; ++y) {
        int yy = y;
        if (!p->walls) yy = wrap(y, ny);
        else if (y < 0 || y >= ny) continue; /* ghost rows filled below */
        for (int x = 0; x < nx; ++x)
            for (int i = 0; i < 9; ++i) {
                const int sx = wrap(x - EX[i], nx);
                int sy = yy - EY[i];
                double fv, gv;
                if (p->walls && (sy < 0 || sy >= ny)) {
                    const size_t src = (size_t)OPP[i] * bn + (size_t)(yy - band_y0) * nx + x;
                    fv = fband[src];
                    gv = gband[src];
                } else {
                    sy = wrap(sy, ny);
                    const int by = sy - band_y0;
                    const size_t src = (size_t)i * bn + (size_t)by * nx + sx;
                    fv = fband[src];
                    gv = gband[src];
                }
                const size_t dst = (size_t)i * rn + (size_t)(y - ry0) * nx + x;
                fs[dst] = fv;
                gs[dst] = gv;
            }
    }
    for (int y = ry0; y < ry1; ++y) {
        if (p->walls && (y < 0 || y >= ny)) continue;
        for (int x = 0; x < nx; ++x) {
            double ph = 0.0;
            for (int i = 0; i < 9; ++i) ph += gs[(size_t)i * rn + (size_t)(y - ry0) * nx + x];
            phi_full[(size_t)(y - ry0) * nx + x] = ph;
        }
    }
    for (int y = y0; y < y1; ++y)
        for (int x = x0; x < x1; ++x) {
            /* Eq. best on the window rows; ghost rows by the wetting rule */
            double sx = 0.0, sy = 0.0, sl = 0.0;
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) {
                    const int qx = wrap(x + c - 1, nx);
                    const int qy = y + r - 1;
                    double v;
                    if (p->walls && qy < 0)
                        v = phi_full[(size_t)(wet_k(p) - 1 - ry0) * nx + qx] -
                            wet_k(p) * p->h_bottom;
                    else if (p->walls && qy >= ny)
                        v = phi_full[(size_t)(ny - wet_k(p) - ry0) * nx + qx] -
                            wet_k(p) * p->h_top;
                    else
                        v = phi_full[(size_t)(qy - ry0) * nx + qx];
                    sx += DX_STENCIL[r][c] * v;
                    sy += DX_STENCIL[c][r] * v;
                    sl += LAP_STENCIL[r][c] * v;
                }
            const double dxv = sx / 12.0, dyv = sy / 12.0, lapv = sl / 6.0;
            const size_t kk = (size_t)(y - ry0) * nx + x;
            double fin[9], gin[9], r = 0.0, jx = 0.0, jy = 0.0;
            for (int i = 0; i < 9; ++i) {
                fin[i] = fs[(size_t)i * rn + kk];
                gin[i] = gs[(size_t)i * rn + kk];
                r += fin[i];
                jx += fin[i] * EX[i];
                jy += fin[i] * EY[i];
            }
            const double ph = phi_full[kk];
            double ueqx = jx / r, ueqy = jy / r;
            const int step2_node = p->zero_u_at_walls && is_boundary_node(p, ny, y);
            if (step2_node) {
                ueqx = 0.0;
                ueqy = 0.0;
            }
            double feq[9], geq[9], fo[9];
            orc_node_equilibrium(p, r, ph, ueqx, ueqy, dxv, dyv, lapv, feq, geq);
            const double tau = orc_node_tau(p, ph);
            collide_f(p, minv, fin, feq, 1.0 / tau, step2_node, fo);
            const size_t wk = (size_t)(y - y0) * wx + (x - x0);
            for (int i = 0; i < 9; ++i) {
                fout_w[(size_t)i * wx * wy + wk] = fo[i];
                gout_w[(size_t)i * wx * wy + wk] = gin[i] - (gin[i] - geq[i]) / p->tau_phi;
            }
        }
    free(fs);
    free(gs);
    free(phi_full);
    return 0;
}

/* ============================================================ geometry */
/* Solid obstacles inside the lattice (capillary filling, Sec. VI).
 *
 * cls[y*nx + x] = 0 marks a fluid node and k in 1..7 a solid node of
 * wetting class k, whose inward-normal wetting gradient is hcls[k].  With
 * walls == 1 the rows y = -1 and y = ny are solid as well, with h_bottom and
 * h_top.  Solid nodes carry no fluid: their populations are never streamed
 * from or collided.
 *
 * Readings (the paper states the wetting condition only for a flat wall):
 *  - bounce-back: a population whose pull source r - e_i is solid is the
 *    node's own reversed post-collision population (mid-link, as for walls);
 *  - Step-2 boundary nodes: fluid nodes with a solid node among their eight
 *    neighbours;
 *  - wetting ghost value of a solid node s next to fluid: the mirror rule of
 *    the flat wall applied along each axis direction d in which s + d is
 *    fluid, averaged: phi(s) = mean_d phi(s + 2d) - 2 h(s) (one-sided rule:
 *    mean_d phi(s + d) - h(s)).  If no axis
 *    neighbour is fluid (s touches fluid through a corner only) the
 *    diagonal directions are used the same way.  Every mirror node s + 2d
 *    must be fluid (features at least two nodes thick); otherwise the
 *    geometry is rejected.
 * On an obstacle-free lattice this is exactly the ghost-row rule above.
 *
 * Node bounce-back (Fig. 4b: the wall lies on the boundary nodes; the paper
 * gives no more), class ORC_NODE_WALL in row 0 or row ny - 1 of a walled
 * lattice.  Read as the full-way scheme:
 *  - a wall node streams like a fluid node (its pulls from beyond the
 *    lattice take its own opposite population, as at a mid-link wall) and,
 *    instead of colliding, reverses every population: f'_i = f_opp(i), the
 *    same for g;
 *  - for the stencils of its fluid neighbours its phi is the one-sided
 *    wetting value across one spacing from the first fluid row,
 *    phi(x, 0) = phi(x, 1) - h_bottom (phi(x, ny-1) = phi(x, ny-2) - h_top);
 *  - fluid nodes next to a wall node are Step-2 boundary nodes;
 *  - it carries no fluid of its own (its moments are not reported), but
 *    its populations are part of the conserved totals;
 *  - initially it holds the rest equilibrium of its wetting phi value. */
#define ORC_NODE_WALL 8

static int geo_node_wall(int nx, int ny, const unsigned char* cls, int x, int y)
{
    if (y < 0 || y >= ny) return 0;
    return cls[(size_t)y * nx + wrap(x, nx)] == ORC_NODE_WALL;
}

static int geo_solid(const orc_params* p, int nx, int ny, const unsigned char* cls, int x, int y)
{
    if (p->walls && (y < 0 || y >= ny)) return 1;
    x = wrap(x, nx);
    y = wrap(y, ny);
    const unsigned char c = cls[(size_t)y * nx + x];
    return c != 0 && c != ORC_NODE_WALL;
}

static double geo_h(const orc_params* p, int nx, int ny, const unsigned char* cls,
                    const double* hcls, int x, int y)
{
    if (p->walls && y < 0) return p->h_bottom;
    if (p->walls && y >= ny) return p->h_top;
    return hcls[cls[(size_t)wrap(y, ny) * nx + wrap(x, nx)]];
}

/* Is (x, y) a fluid node (neither solid nor a wall node)? */
static int geo_fluid(const orc_params* p, int nx, int ny, const unsigned char* cls, int x, int y)
{
    return !geo_solid(p, nx, ny, cls, x, y) && !geo_node_wall(nx, ny, cls, x, y);
}

/* Mirror directions of solid node (x, y): axis directions with a fluid
 * neighbour, else diagonal ones.  Returns how many (0: no fluid neighbour). */
static int geo_mirror_dirs(const orc_params* p, int nx, int ny, const unsigned char* cls,
                           int x, int y, int dirs[4][2])
{
    static const int AX[4][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}};
    static const int DG[4][2] = {{1, 1}, {-1, -1}, {-1, 1}, {1, -1}};
    int n = 0;
    for (int k = 0; k < 4; ++k)
        if (geo_fluid(p, nx, ny, cls, x + AX[k][0], y + AX[k][1])) {
            dirs[n][0] = AX[k][0];
            dirs[n][1] = AX[k][1];
            ++n;
        }
    if (n > 0) return n;
    for (int k = 0; k < 4; ++k)
        if (geo_fluid(p, nx, ny, cls, x + DG[k][0], y + DG[k][1])) {
            dirs[n][0] = DG[k][0];
            dirs[n][1] = DG[k][1];
            ++n;
        }
    return n;
}

/* 0 if every solid node next to fluid has fluid mirror nodes, -1 if not,
 * -2 if a class index is out of range. */
int orc_geo_check(const orc_params* p, int nx, int ny, const unsigned char* cls)
{
    for (int y = -1; y <= ny; ++y) {
        if (!p->walls && (y < 0 || y >= ny)) continue;
        for (int x = 0; x < nx; ++x) {
            if (y >= 0 && y < ny && cls[(size_t)y * nx + x] == ORC_NODE_WALL) {
                /* node walls: outermost rows of a walled lattice of >= 4 rows,
                 * with fluid in the rows next to them */
                if (!p->walls || (y != 0 && y != ny - 1) || ny < 4) return -2;
                if (cls[(size_t)(y == 0 ? 1 : ny - 2) * nx + x] != 0) return -1;
                continue;
            }
            if (y >= 0 && y < ny && cls[(size_t)y * nx + x] > 7) return -2;
            if (!geo_solid(p, nx, ny, cls, x, y)) continue;
            int dirs[4][2];
            const int n = geo_mirror_dirs(p, nx, ny, cls, x, y, dirs);
            for (int k = 0; k < n; ++k) {
                const int mx = x + 2 * dirs[k][0], my = y + 2 * dirs[k][1];
                if (geo_solid(p, nx, ny, cls, mx, my)) return -1;
                /* an obstacle's mirror node must be fluid, not a node wall
                 * (the rows beyond a node wall are never mirrored) */
                if (y >= 0 && y < ny && geo_node_wall(nx, ny, cls, mx, my)) return -1;
            }
        }
    }
    return 0;
}

/* phi at (x, y), x periodic, y periodic or walled, with the ghost rule at
 * solid nodes.  Only called for nodes next to fluid. */
static double geo_phi_at(const orc_params* p, int nx, int ny, const unsigned char* cls,
                         const double* hcls, const double* phi, int x, int y)
{
    if (geo_node_wall(nx, ny, cls, x, y)) {
        const int in = y == 0 ? 1 : ny - 2; /* the first fluid row */
        return phi[(size_t)in * nx + wrap(x, nx)] - (y == 0 ? p->h_bottom : p->h_top);
    }
    if (!geo_solid(p, nx, ny, cls, x, y))
        return phi[(size_t)wrap(y, ny) * nx + wrap(x, nx)];
    int dirs[4][2];
    const int n = geo_mirror_dirs(p, nx, ny, cls, x, y, dirs);
    double sum = 0.0;
    const int m = wet_k(p);
    for (int k = 0; k < n; ++k) {
        const int mx = x + m * dirs[k][0], my = y + m * dirs[k][1];
        sum += phi[(size_t)wrap(my, ny) * nx + wrap(mx, nx)];
    }
    return sum / n - m * geo_h(p, nx, ny, cls, hcls, x, y);
}

/* Eq. best at every fluid node with the ghost rule at solid neighbours;
 * solid nodes get 0. */
void orc_phi_derivatives_geo(const orc_params* p, int nx, int ny, const unsigned char* cls,
                             const double* hcls, const double* phi, double* dx, double* dy,
                             double* lap)
{
    int y;
#pragma omp parallel for num_threads(orc_get_threads()) schedule(static)
    for (y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            const size_t k = (size_t)y * nx + x;
            dx[k] = dy[k] = lap[k] = 0.0;
            if (cls[k] != 0) continue;
            double sx = 0.0, sy = 0.0, sl = 0.0;
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) {
                    const double v = geo_phi_at(p, nx, ny, cls, hcls, phi, x + c - 1, y + r - 1);
                    sx += DX_STENCIL[r][c] * v;
                    sy += DX_STENCIL[c][r] * v;
                    sl += LAP_STENCIL[r][c] * v;
                }
            dx[k] = sx / 12.0;
            dy[k] = sy / 12.0;
            lap[k] = sl / 6.0;
        }
}

/* Initial populations with obstacles: fluid nodes as orc_init (with the
 * ghost rule), solid nodes at rest with no order parameter (f = w, g = 0). */
int orc_init_geo(const orc_params* p, int nx, int ny, const unsigned char* cls,
                 const double* hcls, const double* phi0, double* f, double* g)
{
    if (orc_geo_check(p, nx, ny, cls) != 0) return -1;
    static const double T[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                                1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
    const size_t n = (size_t)nx * ny;
    double* dx = malloc(n * sizeof(double));
    double* dy = malloc(n * sizeof(double));
    double* lap = malloc(n * sizeof(double));
    orc_phi_derivatives_geo(p, nx, ny, cls, hcls, phi0, dx, dy, lap);
    for (size_t k = 0; k < n; ++k) {
        double feq[9], geq[9];
        if (cls[k] == ORC_NODE_WALL) {
            const int y = (int)(k / nx), x = (int)(k % nx);
            const double pw = geo_phi_at(p, nx, ny, cls, hcls, phi0, x, y);
            orc_node_equilibrium(p, 1.0, pw, 0.0, 0.0, 0.0, 0.0, 0.0, feq, geq);
        } else if (cls[k] != 0) {
            for (int i = 0; i < 9; ++i) {
                feq[i] = T[i];
                geq[i] = 0.0;
            }
        } else {
            orc_node_equilibrium(p, 1.0, phi0[k], 0.0, 0.0, dx[k], dy[k], lap[k], feq, geq);
        }
        for (int i = 0; i < 9; ++i) {
            f[(size_t)i * n + k] = feq[i];
            g[(size_t)i * n + k] = geq[i];
        }
    }
    free(dx);
    free(dy);
    free(lap);
    return 0;
}

/* nsteps time steps with obstacles: Steps 1-4 of Sec. V on the fluid
 * nodes, with the readings stated above.  Returns -1 (state untouched) if
 * the geometry is rejected. */
int orc_step_geo(const orc_params* p, int nx, int ny, const unsigned char* cls,
                 const double* hcls, double* f, double* g, int nsteps)
{
    if (orc_geo_check(p, nx, ny, cls) != 0) return -1;
    const size_t n = (size_t)nx * ny;
    double* fs = malloc(9 * n * sizeof(double));
    double* gs = malloc(9 * n * sizeof(double));
    double* rho = calloc(n, sizeof(double));
    double* phi = calloc(n, sizeof(double));
    double* ux = calloc(n, sizeof(double));
    double* uy = calloc(n, sizeof(double));
    double* dx = malloc(n * sizeof(double));
    double* dy = malloc(n * sizeof(double));
    double* lap = malloc(n * sizeof(double));
    double minv[9][9];
    mrt_inverse(minv);

    for (int s = 0; s < nsteps; ++s) {
        /* pull-stream with bounce-back from solid sources (fluid and node-wall
         * nodes) */
        int y;
#pragma omp parallel for num_threads(orc_get_threads()) schedule(static)
        for (y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const size_t k = (size_t)y * nx + x;
                if (cls[k] != 0 && cls[k] != ORC_NODE_WALL) continue;
                for (int i = 0; i < 9; ++i) {
                    const int sx = x - EX[i], sy = y - EY[i];
                    size_t src;
                    int pop;
                    if (geo_solid(p, nx, ny, cls, sx, sy)) {
                        src = k;
                        pop = OPP[i];
                    } else {
                        src = (size_t)wrap(sy, ny) * nx + wrap(sx, nx);
                        pop = i;
                    }
                    fs[(size_t)i * n + k] = f[(size_t)pop * n + src];
                    gs[(size_t)i * n + k] = g[(size_t)pop * n + src];
                }
            }

        /* Step 1: Eq. moments on fluid nodes */
        long long k;
#pragma omp parallel for num_threads(orc_get_threads()) schedule(static)
        for (k = 0; k < (long long)n; ++k) {
            if (cls[k] != 0) continue;
            double r = 0.0, ph = 0.0, jx = 0.0, jy = 0.0;
            for (int i = 0; i < 9; ++i) {
                const double fi = fs[(size_t)i * n + k];
                r += fi;
                jx += fi * EX[i];
                jy += fi * EY[i];
                ph += gs[(size_t)i * n + k];
            }
            rho[k] = r;
            phi[k] = ph;
            ux[k] = jx / r;
            uy[k] = jy / r;
        }

        /* Eq. best with the ghost rule at solid neighbours */
        orc_phi_derivatives_geo(p, nx, ny, cls, hcls, phi, dx, dy, lap);

        /* Step 2, equilibria, Step 3 collision */
#pragma omp parallel for num_threads(orc_get_threads()) schedule(static)
        for (y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const size_t kk = (size_t)y * nx + x;
                if (cls[kk] == ORC_NODE_WALL) {
                    /* node bounce-back: every population reversed */
                    for (int i = 0; i < 9; ++i) {
                        f[(size_t)i * n + kk] = fs[(size_t)OPP[i] * n + kk];
                        g[(size_t)i * n + kk] = gs[(size_t)OPP[i] * n + kk];
                    }
                    continue;
                }
                if (cls[kk] != 0) continue;
                int next_to_solid = 0;
                for (int i = 1; i < 9; ++i)
                    if (geo_solid(p, nx, ny, cls, x + EX[i], y + EY[i]) ||
                        geo_node_wall(nx, ny, cls, x + EX[i], y + EY[i]))
                        next_to_solid = 1;
                const int step2_node = p->zero_u_at_walls && next_to_solid;
                double ueqx = ux[kk], ueqy = uy[kk];
                if (step2_node) {
                    ueqx = 0.0;
                    ueqy = 0.0;
                }
                double feq[9], geq[9], fin[9], fout[9];
                orc_node_equilibrium(p, rho[kk], phi[kk], ueqx, ueqy, dx[kk], dy[kk], lap[kk],
                                     feq, geq);
                const double tau = orc_node_tau(p, phi[kk]);
                for (int i = 0; i < 9; ++i) fin[i] = fs[(size_t)i * n + kk];
                collide_f(p, minv, fin, feq, 1.0 / tau, step2_node, fout);
                for (int i = 0; i < 9; ++i) {
                    f[(size_t)i * n + kk] = fout[i];
                    const double gi = gs[(size_t)i * n + kk];
                    g[(size_t)i * n + kk] = gi - (gi - geq[i]) / p->tau_phi; /* Eq. gevo */
                }
            }
    }
    free(fs);
    free(gs);
    free(rho);
    free(phi);
    free(ux);
    free(uy);
    free(dx);
    free(dy);
    free(lap);
    return 0;
}
