/*
 * Plain FP64 CPU oracle for the anisotropic-equilibrium BGK lattice Boltzmann method
 * (Kruger, Weinmiller, Latz, Danner: "Lattice Boltzmann Methods with Anisotropic Equilibrium
 * Distributions").
 *
 * TEST INFRASTRUCTURE ONLY. The test suite, the smoke check and the CPU-baseline leg of the
 * benchmark are the only callers. It shares no code, header, table or helper with the CUDA
 * library: lattices are re-derived here from the Gauss-Hermite quadrature, the equilibrium is the
 * paper's tensor form written as full index contractions, streaming is the push form
 * (collide, then move), and populations are stored cell-major (AoS). It is deliberately slow.
 *
 * Conventions shared with the library's public interface (and nothing else):
 *   cell index  n = x + nx*(y + ny*z); fields rho[N], u[d][N]; Theta is d*d row-major;
 *   Pi components in the order xx, yy, (zz), xy, (xz, yz); dTheta in the same order.
 *   Theta := c_s^2 A^{-1} (second moment of the equilibrium, Appendix E), K~ := c_s^2 K
 *   = Theta - c_s^2 I (Eq. K-term); the code's velocity u is the paper's lattice velocity s.
 *
 * Parity status of each function (what pins it) is listed in the header comment of each.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define MAXQ 27
#define CS2 (1.0 / 3.0)

typedef struct {
    int d, q;
    int c[MAXQ][3];
    double w[MAXQ];
    int opp[MAXQ];
    /* Hermite tensors of each lattice velocity (see hermite_tensors), filled once per lattice */
    double H1[MAXQ][3], H2[MAXQ][3][3], H3[MAXQ][3][3][3];
} olat;

static void hermite_tensors(const olat* L, int i, double H1[3], double H2[3][3], double H3[3][3][3]);

/* ---------------------------------------------------------------------------------------------
 * Lattices (Appendix C). D1Q3 nodes are the roots of the probabilists' Hermite polynomial
 * H3(x) = x^3 - 3x, weights w_i = n!/[n H2(x_i)]^2 with H2(x) = x^2 - 1 (Eq. weights); lattice
 * velocities follow from the rescaling c_i = c_s v_i with c_s^2 = 1/3 (Sec. 2.3). D2Q9 and D3Q27
 * are tensor products of D1Q3. D3Q19 is the symmetry-reduced set the paper takes from Shan et al.
 * (Appendix C): every c in {-1,0,1}^3 with |c|^2 <= 2, textbook weights 1/3, 1/18, 1/36.
 * Pinned by: printed D1Q3 nodes/weights, sum w = 1, second- and fourth-order isotropy.
 * ------------------------------------------------------------------------------------------- */
static double hermite_prob(int n, double x) {
    /* H0 = 1, H1 = x, H_{n+1} = x H_n - n H_{n-1} (probabilists' recursion, Appendix B) */
    double h0 = 1.0, h1 = x;
    if (n == 0) return h0;
    for (int k = 1; k < n; ++k) {
        double h2 = x * h1 - (double)k * h0;
        h0 = h1;
        h1 = h2;
    }
    return h1;
}

/* D1Q3 nodes x_k (roots of H3) and Gauss-Hermite weights w_k. */
void oracle_d1q3(double* nodes, double* weights) {
    const int n = 3;
    double roots[3] = {0.0, sqrt(3.0), -sqrt(3.0)}; /* x^3 - 3x = x (x^2 - 3) */
    double nfact = 6.0;
    for (int k = 0; k < 3; ++k) {
        double h = (double)n * hermite_prob(n - 1, roots[k]);
        nodes[k] = roots[k];
        weights[k] = nfact / (h * h);
    }
}

static int build_lattice(int q, olat* L) {
    double nodes[3], w1[3];
    oracle_d1q3(nodes, w1);
    int cint[3];
    double wint[3];
    for (int k = 0; k < 3; ++k) {
        cint[k] = (int)lround(nodes[k] * sqrt(CS2)); /* c = c_s v */
        wint[k] = w1[k];
    }
    memset(L, 0, sizeof(*L));
    if (q == 9) {
        L->d = 2;
        int n = 0;
        for (int b = 0; b < 3; ++b)
            for (int a = 0; a < 3; ++a) {
                L->c[n][0] = cint[a];
                L->c[n][1] = cint[b];
                L->c[n][2] = 0;
                L->w[n] = wint[a] * wint[b];
                ++n;
            }
        L->q = n;
    } else if (q == 27) {
        L->d = 3;
        int n = 0;
        for (int g = 0; g < 3; ++g)
            for (int b = 0; b < 3; ++b)
                for (int a = 0; a < 3; ++a) {
                    L->c[n][0] = cint[a];
                    L->c[n][1] = cint[b];
                    L->c[n][2] = cint[g];
                    L->w[n] = wint[a] * wint[b] * wint[g];
                    ++n;
                }
        L->q = n;
    } else if (q == 19) {
        L->d = 3;
        int n = 0;
        for (int g = 0; g < 3; ++g)
            for (int b = 0; b < 3; ++b)
                for (int a = 0; a < 3; ++a) {
                    int cx = cint[a], cy = cint[b], cz = cint[g];
                    int c2 = cx * cx + cy * cy + cz * cz;
                    if (c2 > 2) continue;
                    L->c[n][0] = cx;
                    L->c[n][1] = cy;
                    L->c[n][2] = cz;
                    L->w[n] = (c2 == 0) ? 1.0 / 3.0 : (c2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
                    ++n;
                }
        L->q = n;
    } else {
        return -1;
    }
    for (int i = 0; i < L->q; ++i) hermite_tensors(L, i, L->H1[i], L->H2[i], L->H3[i]);
    for (int i = 0; i < L->q; ++i) {
        L->opp[i] = -1;
        for (int j = 0; j < L->q; ++j)
            if (L->c[j][0] == -L->c[i][0] && L->c[j][1] == -L->c[i][1] && L->c[j][2] == -L->c[i][2])
                L->opp[i] = j;
    }
    return 0;
}

/* Export the oracle's own velocity set (its own ordering), weights and opposite map. */
int oracle_lattice(int q, int* c, double* w, int* opp) {
    olat L;
    if (build_lattice(q, &L)) return -1;
    for (int i = 0; i < L.q; ++i) {
        for (int a = 0; a < 3; ++a) c[3 * i + a] = L.c[i][a];
        w[i] = L.w[i];
        opp[i] = L.opp[i];
    }
    return L.q;
}

/* K~ = Theta - c_s^2 I, embedded in 3x3. */
static void ktilde(const olat* L, const double* Theta, double Kt[3][3]) {
    int d = L->d;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Kt[a][b] = 0.0;
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) Kt[a][b] = Theta[a * d + b] - (a == b ? CS2 : 0.0);
}

static inline double kd(int a, int b) { return a == b ? 1.0 : 0.0; }

/* Hermite tensors of the rescaled velocity (Eq. 3rd_order_equilibrium, lattice units):
 * H1_a = c_a, H2_ab = c_a c_b - c_s^2 d_ab,
 * H3_abg = c_a c_b c_g - c_s^2 (c_a d_bg + c_b d_ga + c_g d_ab). */
static void hermite_tensors(const olat* L, int i, double H1[3], double H2[3][3], double H3[3][3][3]) {
    double c[3] = {L->c[i][0], L->c[i][1], L->c[i][2]};
    int d = L->d;
    for (int a = 0; a < 3; ++a) {
        H1[a] = (a < d) ? c[a] : 0.0;
        for (int b = 0; b < 3; ++b) {
            H2[a][b] = (a < d && b < d) ? c[a] * c[b] - CS2 * kd(a, b) : 0.0;
            for (int g = 0; g < 3; ++g)
                H3[a][b][g] = (a < d && b < d && g < d)
                                  ? c[a] * c[b] * c[g] - CS2 * (c[a] * kd(b, g) + c[b] * kd(g, a) + c[g] * kd(a, b))
                                  : 0.0;
        }
    }
}

/* ---------------------------------------------------------------------------------------------
 * Discrete anisotropic equilibrium, Eq. (3rd_order_equilibrium) with Eq. (feq_i):
 *   feq_i = w_i rho [ 1 + a1.H1/c_s^2 + a2:H2/(2 c_s^4) + a3:H3/(6 c_s^6) ],
 *   a1 = u, a2_ab = u_a u_b + K~_ab, a3_abg = u_a u_b u_g + K~_ab u_g + K~_bg u_a + K~_ga u_b
 * (Appendix B coefficients in lattice units). order = 2 drops the a3 term (Sec. 2.2 / Sec. 4).
 * Pinned by: exact discrete moments rho, rho u, rho(Theta + uu) on all lattices, the mixed third
 * moments on the tensor-product lattices (Appendix E, exact by Appendix C's degree argument),
 * and the reduction to the textbook isotropic equilibrium at Theta = c_s^2 I.
 * ------------------------------------------------------------------------------------------- */
static void feq_cell(const olat* L, int order, double rho, const double u3[3], double Kt[3][3], double* feq) {
    double a2[3][3], a3[3][3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            a2[a][b] = u3[a] * u3[b] + Kt[a][b];
            for (int g = 0; g < 3; ++g)
                a3[a][b][g] = u3[a] * u3[b] * u3[g] + Kt[a][b] * u3[g] + Kt[b][g] * u3[a] + Kt[g][a] * u3[b];
        }
    for (int i = 0; i < L->q; ++i) {
        const double* H1 = L->H1[i];
        const double(*H2)[3] = L->H2[i];
        const double(*H3)[3][3] = L->H3[i];
        double s1 = 0.0, s2 = 0.0, s3 = 0.0;
        for (int a = 0; a < 3; ++a) {
            s1 += u3[a] * H1[a];
            for (int b = 0; b < 3; ++b) {
                s2 += a2[a][b] * H2[a][b];
                for (int g = 0; g < 3; ++g) s3 += a3[a][b][g] * H3[a][b][g];
            }
        }
        double p = 1.0 + s1 / CS2 + s2 / (2.0 * CS2 * CS2);
        if (order >= 3) p += s3 / (6.0 * CS2 * CS2 * CS2);
        feq[i] = L->w[i] * rho * p;
    }
}

/* One-cell equilibrium for tests: feq[q] in the oracle's own direction order. */
int oracle_feq(int q, double rho, const double* u, const double* Theta, int order, double* feq) {
    olat L;
    if (build_lattice(q, &L)) return -1;
    double Kt[3][3];
    ktilde(&L, Theta, Kt);
    double u3[3] = {0, 0, 0};
    for (int a = 0; a < L.d; ++a) u3[a] = u[a];
    feq_cell(&L, order, rho, u3, Kt, feq);
    return 0;
}

/* Periodic neighbour of cell (x,y,z) along integer offset (dx,dy,dz). */
static inline int64_t neighbour(int nx, int ny, int nz, int x, int y, int z, int dx, int dy, int dz) {
    int xx = ((x + dx) % nx + nx) % nx;
    int yy = ((y + dy) % ny + ny) % ny;
    int zz = ((z + dz) % nz + nz) % nz;
    return (int64_t)xx + (int64_t)nx * ((int64_t)yy + (int64_t)ny * zz);
}

static inline int is_solid(const uint8_t* solid, int64_t n) { return solid != NULL && solid[n] != 0; }

/* Moments of one cell: rho = sum f_i, j = sum f_i c_i (Eqs. a0discrete_f, a1discrete_f). */
static void cell_moments(const olat* L, const double* f, double* rho, double u3[3]) {
    double r = 0.0, j[3] = {0, 0, 0};
    for (int i = 0; i < L->q; ++i) {
        r += f[i];
        for (int a = 0; a < 3; ++a) j[a] += f[i] * L->c[i][a];
    }
    *rho = r;
    for (int a = 0; a < 3; ++a) u3[a] = j[a] / r;
}

/* ---------------------------------------------------------------------------------------------
 * Initial state f_i(x, 0) = feq_i(rho0(x), u0(x)) at fluid cells, zero at solid cells
 * (Sec. 4 initialises from the velocity and density fields). f is [N][q], oracle order.
 * ------------------------------------------------------------------------------------------- */
int oracle_init(int q, int nx, int ny, int nz, const double* Theta, int order, const uint8_t* solid,
                const double* rho0, const double* u0, double* f) {
    olat L;
    if (build_lattice(q, &L)) return -1;
    double Kt[3][3];
    ktilde(&L, Theta, Kt);
    int64_t N = (int64_t)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        double* fn = f + n * L.q;
        if (is_solid(solid, n)) {
            for (int i = 0; i < L.q; ++i) fn[i] = 0.0;
            continue;
        }
        double u3[3] = {0, 0, 0};
        for (int a = 0; a < L.d; ++a) u3[a] = u0[(int64_t)a * N + n];
        feq_cell(&L, order, rho0[n], u3, Kt, fn);
    }
    return 0;
}

/* ---------------------------------------------------------------------------------------------
 * One time step of the fully discrete BGK LBE (Eq. LBE_BGK) with dt = 1:
 *   collide  f*_i(x) = f_i(x) + (feq_i(x) - f_i(x)) / tau,
 *   stream   f_i(x + c_i, t+1) = f*_i(x)              if x + c_i is fluid (periodic wrap),
 *            f_{opp(i)}(x, t+1) = f*_i(x)             otherwise (half-way bounce-back, wall at
 *                                                      rest half-way along the link).
 * The paper defers the space-time discretisation to the textbook (Sec. 2.3) and names bounce-back
 * only as future work (Sec. 5); the wall rule is the textbook half-way bounce-back.
 * Pinned by: pure streaming at tau -> infinity, fixed points, conservation, linear decay rates.
 * ------------------------------------------------------------------------------------------- */
static void step_push(const olat* L, int nx, int ny, int nz, double tau, double Kt[3][3], int order,
                      const uint8_t* solid, const double* f, double* fn) {
    int64_t N = (int64_t)nx * ny * nz;
    int q = L->q;
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        if (is_solid(solid, n)) continue;
        int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((int64_t)nx * ny));
        const double* fc = f + n * q;
        double rho, u3[3];
        cell_moments(L, fc, &rho, u3);
        double feq[MAXQ];
        feq_cell(L, order, rho, u3, Kt, feq);
        for (int i = 0; i < q; ++i) {
            double fs = fc[i] + (feq[i] - fc[i]) / tau;
            int64_t m = neighbour(nx, ny, nz, x, y, z, L->c[i][0], L->c[i][1], L->c[i][2]);
            if (!is_solid(solid, m))
                fn[m * q + i] = fs;
            else
                fn[n * q + L->opp[i]] = fs;
        }
    }
}

/* Post-collision populations of one cell (oracle order): f*_i = f_i + (feq_i(m(f)) - f_i)/tau. */
int oracle_collide_cell(int q, double tau, const double* Theta, int order, const double* f, double* fs) {
    olat L;
    if (build_lattice(q, &L)) return -1;
    double Kt[3][3];
    ktilde(&L, Theta, Kt);
    double rho, u3[3], feq[MAXQ];
    cell_moments(&L, f, &rho, u3);
    feq_cell(&L, order, rho, u3, Kt, feq);
    for (int i = 0; i < L.q; ++i) fs[i] = f[i] + (feq[i] - f[i]) / tau;
    return 0;
}

/* Advance f ([N][q], in place) by nsteps. */
int oracle_run(int q, int nx, int ny, int nz, double tau, const double* Theta, int order, const uint8_t* solid,
               double* f, int nsteps) {
    olat L;
    if (build_lattice(q, &L)) return -1;
    double Kt[3][3];
    ktilde(&L, Theta, Kt);
    int64_t N = (int64_t)nx * ny * nz;
    double* g = (double*)calloc((size_t)N * L.q, sizeof(double));
    if (!g) return -2;
    double* a = f;
    double* b = g;
    for (int s = 0; s < nsteps; ++s) {
        memset(b, 0, (size_t)N * L.q * sizeof(double));
        step_push(&L, nx, ny, nz, tau, Kt, order, solid, a, b);
        double* t = a;
        a = b;
        b = t;
    }
    if (a != f) memcpy(f, a, (size_t)N * L.q * sizeof(double));
    free(g);
    return 0;
}

/* ---------------------------------------------------------------------------------------------
 * Observables of the pre-collision state (Eqs. a0discrete_f, a1discrete_f; second moment as in
 * Appendix E): rho, u = j/rho, Pi_ab = sum_i f_i c_ia c_ib. Solid cells report zeros.
 * Any output pointer may be NULL.
 * ------------------------------------------------------------------------------------------- */
int oracle_moments(int q, int nx, int ny, int nz, const uint8_t* solid, const double* f, double* rho, double* u,
                   double* Pi) {
    olat L;
    if (build_lattice(q, &L)) return -1;
    int64_t N = (int64_t)nx * ny * nz;
    int d = L.d;
    int np = d == 2 ? 3 : 6;
    int pa[6], pb[6];
    if (d == 2) {
        int A[3] = {0, 1, 0}, B[3] = {0, 1, 1};
        for (int k = 0; k < 3; ++k) pa[k] = A[k], pb[k] = B[k];
    } else {
        int A[6] = {0, 1, 2, 0, 0, 1}, B[6] = {0, 1, 2, 1, 2, 2};
        for (int k = 0; k < 6; ++k) pa[k] = A[k], pb[k] = B[k];
    }
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        const double* fc = f + n * L.q;
        double r = 0.0, u3[3] = {0, 0, 0}, P[6] = {0, 0, 0, 0, 0, 0};
        if (!is_solid(solid, n)) {
            cell_moments(&L, fc, &r, u3);
            for (int k = 0; k < np; ++k)
                for (int i = 0; i < L.q; ++i) P[k] += fc[i] * L.c[i][pa[k]] * L.c[i][pb[k]];
        } else {
            u3[0] = u3[1] = u3[2] = 0.0;
        }
        if (rho) rho[n] = r;
        if (u)
            for (int a = 0; a < d; ++a) u[(int64_t)a * N + n] = u3[a];
        if (Pi)
            for (int k = 0; k < np; ++k) Pi[(int64_t)k * N + n] = P[k];
    }
    return 0;
}

/* Total mass and momentum over fluid cells, Kahan-compensated FP64 sums (Sec. 3, continuity and
 * momentum balance). out[0] = sum rho, out[1..d] = sum j. */
int oracle_totals(int q, int nx, int ny, int nz, const uint8_t* solid, const double* f, double* out) {
    olat L;
    if (build_lattice(q, &L)) return -1;
    int64_t N = (int64_t)nx * ny * nz;
    double s[4] = {0, 0, 0, 0}, c[4] = {0, 0, 0, 0};
    for (int64_t n = 0; n < N; ++n) {
        if (is_solid(solid, n)) continue;
        const double* fc = f + n * L.q;
        double v[4] = {0, 0, 0, 0};
        for (int i = 0; i < L.q; ++i) {
            v[0] += fc[i];
            for (int a = 0; a < 3; ++a) v[1 + a] += fc[i] * L.c[i][a];
        }
        for (int k = 0; k < 4; ++k) {
            double y = v[k] - c[k];
            double t = s[k] + y;
            c[k] = (t - s[k]) - y;
            s[k] = t;
        }
    }
    for (int k = 0; k <= L.d; ++k) out[k] = s[k];
    return 0;
}

/* ---------------------------------------------------------------------------------------------
 * Discrete adjoint of the map  u(T) <- f(T) <- ... <- f(0) = feq(rho0, u0; Theta)  (reverse mode
 * of the LBE above, written from the chain rule; the paper has no adjoint). The whole trajectory
 * is stored, so this is for small grids only.
 *   seed      lambda_T,i = sum_a g_a (c_ia - u_a)/rho                 (du_a/df_i)
 *   reverse   mu_i(x)   = lambda_{t+1,i}(x + c_i), or lambda_{t+1,opp i}(x) when x + c_i is solid
 *             lambda_t  = J_C(f_t)^T mu with J_C,ij = (1-1/tau) d_ij + (1/tau) dfeq_i/df_j and
 *             dfeq_i/df_j = feq_i/rho + sum_a dfeq_i/du_a (c_ja - u_a)/rho   (chain rule via u)
 *   params    dL/dtau  += sum_i mu_i * (-(feq_i - f_i)/tau^2)
 *             dL/dK~ab += (1/tau) sum_i mu_i dfeq_i/dK~ab, plus sum_i lambda_0,i dfeq_i/dK~ab
 *             at the initial equilibrium; dTheta = dK~, symmetrised (off-diagonal = ab + ba).
 *   init      dL/du0_a(x) = sum_i lambda_0,i(x) dfeq_i/du_a(rho0(x), u0(x)).
 * All derivatives are taken of the tensor form by differentiating a2 and a3 entry by entry.
 * Pinned by: central finite differences of oracle_run (tests).
 * ------------------------------------------------------------------------------------------- */
static void feq_derivs(const olat* L, int order, double rho, const double u3[3], double Kt[3][3], double* feq,
                       double dU[MAXQ][3], double dK[MAXQ][3][3]) {
    feq_cell(L, order, rho, u3, Kt, feq);
    double a2[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) a2[a][b] = u3[a] * u3[b] + Kt[a][b];
    (void)a2;
    for (int i = 0; i < L->q; ++i) {
        const double* H1 = L->H1[i];
        const double(*H2)[3] = L->H2[i];
        const double(*H3)[3][3] = L->H3[i];
        /* d/du_e of s1, s2, s3 */
        for (int e = 0; e < 3; ++e) {
            double ds1 = H1[e];
            double ds2 = 0.0, ds3 = 0.0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    double da2 = kd(a, e) * u3[b] + u3[a] * kd(b, e);
                    ds2 += da2 * H2[a][b];
                    for (int g = 0; g < 3; ++g) {
                        double da3 = kd(a, e) * u3[b] * u3[g] + u3[a] * kd(b, e) * u3[g] + u3[a] * u3[b] * kd(g, e) +
                                     Kt[a][b] * kd(g, e) + Kt[b][g] * kd(a, e) + Kt[g][a] * kd(b, e);
                        ds3 += da3 * H3[a][b][g];
                    }
                }
            double dp = ds1 / CS2 + ds2 / (2.0 * CS2 * CS2);
            if (order >= 3) dp += ds3 / (6.0 * CS2 * CS2 * CS2);
            dU[i][e] = L->w[i] * rho * dp;
        }
        /* d/dK~_ef (unsymmetrised) */
        for (int e = 0; e < 3; ++e)
            for (int f = 0; f < 3; ++f) {
                double ds2 = 0.0, ds3 = 0.0;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) {
                        double da2 = kd(a, e) * kd(b, f);
                        ds2 += da2 * H2[a][b];
                        for (int g = 0; g < 3; ++g) {
                            double da3 = kd(a, e) * kd(b, f) * u3[g] + kd(b, e) * kd(g, f) * u3[a] +
                                         kd(g, e) * kd(a, f) * u3[b];
                            ds3 += da3 * H3[a][b][g];
                        }
                    }
                double dp = ds2 / (2.0 * CS2 * CS2);
                if (order >= 3) dp += ds3 / (6.0 * CS2 * CS2 * CS2);
                dK[i][e][f] = L->w[i] * rho * dp;
            }
    }
}

int oracle_adjoint(int q, int nx, int ny, int nz, double tau, const double* Theta, int order, const uint8_t* solid,
                   const double* rho0, const double* u0, int nsteps, const double* dLdu, double* dTheta, double* dtau,
                   double* du0) {
    olat L;
    if (build_lattice(q, &L)) return -1;
    double Kt[3][3];
    ktilde(&L, Theta, Kt);
    const int d = L.d;
    const int64_t N = (int64_t)nx * ny * nz;
    const size_t S = (size_t)N * L.q;
    double* traj = (double*)calloc(S * (size_t)(nsteps + 1), sizeof(double));
    double* lam = (double*)calloc(S, sizeof(double));
    double* lamn = (double*)calloc(S, sizeof(double));
    if (!traj || !lam || !lamn) {
        free(traj);
        free(lam);
        free(lamn);
        return -2;
    }
    oracle_init(q, nx, ny, nz, Theta, order, solid, rho0, u0, traj);
    for (int t = 0; t < nsteps; ++t)
        step_push(&L, nx, ny, nz, tau, Kt, order, solid, traj + S * t, traj + S * (t + 1));

    /* seed from u(T) */
    const double* fT = traj + S * nsteps;
    for (int64_t n = 0; n < N; ++n) {
        if (is_solid(solid, n)) continue;
        double rho, u3[3];
        cell_moments(&L, fT + n * L.q, &rho, u3);
        for (int i = 0; i < L.q; ++i) {
            double s = 0.0;
            for (int a = 0; a < d; ++a) s += dLdu[(int64_t)a * N + n] * (L.c[i][a] - u3[a]) / rho;
            lamn[n * L.q + i] = s;
        }
    }
    double gK[3][3] = {{0}}, gtau = 0.0;
    for (int t = nsteps - 1; t >= 0; --t) {
        const double* ft = traj + S * t;
        memset(lam, 0, S * sizeof(double));
        for (int64_t n = 0; n < N; ++n) {
            if (is_solid(solid, n)) continue;
            int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((int64_t)nx * ny));
            double mu[MAXQ];
            for (int i = 0; i < L.q; ++i) {
                int64_t m = neighbour(nx, ny, nz, x, y, z, L.c[i][0], L.c[i][1], L.c[i][2]);
                mu[i] = !is_solid(solid, m) ? lamn[m * L.q + i] : lamn[n * L.q + L.opp[i]];
            }
            const double* fc = ft + n * L.q;
            double rho, u3[3], feq[MAXQ], dU[MAXQ][3], dK[MAXQ][3][3];
            cell_moments(&L, fc, &rho, u3);
            feq_derivs(&L, order, rho, u3, Kt, feq, dU, dK);
            for (int j = 0; j < L.q; ++j) {
                double s = 0.0;
                for (int i = 0; i < L.q; ++i) {
                    double dfdf = feq[i] / rho;
                    for (int a = 0; a < 3; ++a) dfdf += dU[i][a] * (L.c[j][a] - u3[a]) / rho;
                    double J = (1.0 - 1.0 / tau) * kd(i, j) + (1.0 / tau) * dfdf;
                    s += mu[i] * J;
                }
                lam[n * L.q + j] = s;
            }
            for (int i = 0; i < L.q; ++i) {
                gtau += mu[i] * (-(feq[i] - fc[i]) / (tau * tau));
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) gK[a][b] += (1.0 / tau) * mu[i] * dK[i][a][b];
            }
        }
        double* tmp = lam;
        lam = lamn;
        lamn = tmp;
    }
    /* lamn now holds lambda_0; gradient through f(0) = feq(rho0, u0; Theta) */
    for (int64_t n = 0; n < N; ++n) {
        if (is_solid(solid, n)) {
            if (du0)
                for (int a = 0; a < d; ++a) du0[(int64_t)a * N + n] = 0.0;
            continue;
        }
        double u3[3] = {0, 0, 0};
        for (int a = 0; a < d; ++a) u3[a] = u0[(int64_t)a * N + n];
        double feq[MAXQ], dU[MAXQ][3], dK[MAXQ][3][3];
        feq_derivs(&L, order, rho0[n], u3, Kt, feq, dU, dK);
        for (int a = 0; a < d; ++a) {
            double s = 0.0;
            for (int i = 0; i < L.q; ++i) s += lamn[n * L.q + i] * dU[i][a];
            if (du0) du0[(int64_t)a * N + n] = s;
        }
        for (int i = 0; i < L.q; ++i)
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) gK[a][b] += lamn[n * L.q + i] * dK[i][a][b];
    }
    if (d == 2) {
        dTheta[0] = gK[0][0];
        dTheta[1] = gK[1][1];
        dTheta[2] = gK[0][1] + gK[1][0];
    } else {
        dTheta[0] = gK[0][0];
        dTheta[1] = gK[1][1];
        dTheta[2] = gK[2][2];
        dTheta[3] = gK[0][1] + gK[1][0];
        dTheta[4] = gK[0][2] + gK[2][0];
        dTheta[5] = gK[1][2] + gK[2][1];
    }
    *dtau = gtau;
    free(traj);
    free(lam);
    free(lamn);
    return 0;
}

/* ---------------------------------------------------------------------------------------------
 * Anisotropic advection-diffusion (the transfer named in Sec. 1 and Sec. 5; the paper gives no
 * equations). A scalar phi carried by a prescribed velocity field u(x) has populations g_i with
 * the equilibrium of Eq. (3rd_order_equilibrium) taken with rho -> phi:
 *   sum geq = phi, sum geq c = phi u, sum geq c c = phi (Theta + u u),
 * relaxed by BGK and streamed as in oracle_run (push, half-way bounce-back at solid cells).
 * Chapman-Enskog (as in Sec. 3) then gives d_t phi + div(phi u) = div((tau - 1/2) Theta grad phi).
 * g is [N][q] in the oracle's order; u is [d][N] and stays fixed.
 * Pinned by: mass conservation, uniform fixed point, and the exact linear decay rate of a
 * diffusing mode against the linearised step and the anisotropic diffusion rate.
 * ------------------------------------------------------------------------------------------- */
int oracle_ade_init(int q, int nx, int ny, int nz, const double* Theta, int order, const uint8_t* solid,
                    const double* phi, const double* u, double* g) {
    return oracle_init(q, nx, ny, nz, Theta, order, solid, phi, u, g);
}

int oracle_ade_run(int q, int nx, int ny, int nz, double tau, const double* Theta, int order, const uint8_t* solid,
                   const double* u, double* g, int nsteps) {
    olat L;
    if (build_lattice(q, &L)) return -1;
    double Kt[3][3];
    ktilde(&L, Theta, Kt);
    const int64_t N = (int64_t)nx * ny * nz;
    const int qq = L.q;
    double* h = (double*)calloc((size_t)N * qq, sizeof(double));
    if (!h) return -2;
    double* a = g;
    double* b = h;
    for (int s = 0; s < nsteps; ++s) {
        memset(b, 0, (size_t)N * qq * sizeof(double));
#pragma omp parallel for schedule(static)
        for (int64_t n = 0; n < N; ++n) {
            if (is_solid(solid, n)) continue;
            int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((int64_t)nx * ny));
            const double* gc = a + n * qq;
            double phi = 0.0;
            for (int i = 0; i < qq; ++i) phi += gc[i];
            double u3[3] = {0, 0, 0};
            for (int d = 0; d < L.d; ++d) u3[d] = u[(int64_t)d * N + n];
            double geq[MAXQ];
            feq_cell(&L, order, phi, u3, Kt, geq);
            for (int i = 0; i < qq; ++i) {
                double gs = gc[i] + (geq[i] - gc[i]) / tau;
                int64_t m = neighbour(nx, ny, nz, x, y, z, L.c[i][0], L.c[i][1], L.c[i][2]);
                if (!is_solid(solid, m))
                    b[m * qq + i] = gs;
                else
                    b[n * qq + L.opp[i]] = gs;
            }
        }
        double* t = a;
        a = b;
        b = t;
    }
    if (a != g) memcpy(g, a, (size_t)N * qq * sizeof(double));
    free(h);
    return 0;
}

/* Post-collision scalar populations of one cell (oracle order): g*_i = g_i + (geq_i(phi, u) - g_i)/tau
 * with phi = sum_i g_i and u the cell's advecting velocity (d values). */
int oracle_ade_collide_cell(int q, double tau, const double* Theta, int order, const double* g, const double* u,
                            double* gs) {
    olat L;
    if (build_lattice(q, &L)) return -1;
    double Kt[3][3];
    ktilde(&L, Theta, Kt);
    double phi = 0.0;
    for (int i = 0; i < L.q; ++i) phi += g[i];
    double u3[3] = {0, 0, 0}, geq[MAXQ];
    for (int a = 0; a < L.d; ++a) u3[a] = u[a];
    feq_cell(&L, order, phi, u3, Kt, geq);
    for (int i = 0; i < L.q; ++i) gs[i] = g[i] + (geq[i] - g[i]) / tau;
    return 0;
}

/* phi = sum_i g_i per cell (0 at solid cells). */
int oracle_ade_scalar(int q, int nx, int ny, int nz, const uint8_t* solid, const double* g, double* phi) {
    olat L;
    if (build_lattice(q, &L)) return -1;
    const int64_t N = (int64_t)nx * ny * nz;
    for (int64_t n = 0; n < N; ++n) {
        double s = 0.0;
        if (!is_solid(solid, n))
            for (int i = 0; i < L.q; ++i) s += g[n * L.q + i];
        phi[n] = s;
    }
    return 0;
}

/* Number of OpenMP threads the oracle runs with (1 when built without OpenMP). */
#ifdef _OPENMP
#include <omp.h>
int oracle_threads(void) { return omp_get_max_threads(); }
#else
int oracle_threads(void) { return 1; }
#endif
