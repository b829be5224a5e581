/*
 * FP64 CPU oracle of the PINN-LBM droplet hot path (arXiv 2504.10539).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file.  It is used by the test suite, by the smoke check and by
 * the benchmark's CPU-baseline leg.  It shares no source, header, table or
 * helper with the CUDA path: the D2Q9 tables, the counter-based random number
 * generator, the initial profile, the step, the metrics, the network and the
 * correction are all written out again here, plainly, in double precision.
 *
 * The paper gives the evolution equation (Sec. II-A, Eq. 1), the network
 * signature and architecture (Sec. II-B Eq. 2, Sec. III-B), the coupling loop
 * (Sec. II-C), the metrics (Sec. II-D Eqs. 9-13, Sec. IV-E Eqs. 14-16) and the
 * droplet set-up (Sec. III-A).  It does not give the lattice, the
 * pseudopotential, the force stencil, the forcing scheme or the correction
 * formula; the readings used for those are stated at each function.
 *
 * Layout of population arrays: f[i*N + y*nx + x], i = 0..8, N = nx*ny
 * (direction-major structure of arrays, x fastest).  This is only the
 * exchange format of the oracle; the oracle streams with two lattices.
 *
 * Every loop is a plain loop over cells.  The only parallelism is an OpenMP
 * "parallel for" over rows of per-cell work that writes disjoint outputs;
 * every reduction is a serial loop in cell order, so results do not depend on
 * the number of threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 9
#define ORC_PI 3.14159265358979323846

/* D2Q9 velocity set and weights.  The paper names no lattice; D2Q9 with
 * c_0=(0,0), c_1..4 = (1,0),(0,1),(-1,0),(0,-1), c_5..8 = (1,1),(-1,1),(-1,-1),(1,-1),
 * w = 4/9, 1/9, 1/36 and c_s^2 = 1/3 is the reading used throughout. */
static const int CX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WQ[Q] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

void orc_lattice_tables(int* cx, int* cy, double* w) {
    for (int i = 0; i < Q; ++i) {
        cx[i] = CX[i];
        cy[i] = CY[i];
        w[i] = WQ[i];
    }
}

static int wrap(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

/* ---------------------------------------------------------------------------
 * Counter-based generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014).  The generator's state after
 * k+1 increments of the golden-gamma 0x9E3779B97F4A7C15 is mixed by the
 * published MurmurHash3-style finaliser; output k for seed s is therefore
 * mix(s + (k+1)*gamma), which can be evaluated for any k independently.
 * ------------------------------------------------------------------------- */
uint64_t orc_splitmix64(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Uniform double in [0,1) from the top 53 bits of output k. */
double orc_uniform01(uint64_t seed, uint64_t k) {
    return (double)(orc_splitmix64(seed, k) >> 11) * (1.0 / 9007199254740992.0);
}

/* ---------------------------------------------------------------------------
 * Equilibrium (Sec. II-A, Eq. 1 via the collision operator).  Standard
 * second-order D2Q9 Maxwellian truncation:
 *   f_i^eq = w_i rho (1 + 3 c_i.u + 4.5 (c_i.u)^2 - 1.5 |u|^2).
 * ------------------------------------------------------------------------- */
void orc_equilibrium(double rho, double ux, double uy, double* feq) {
    double usq = ux * ux + uy * uy;
    for (int i = 0; i < Q; ++i) {
        double cu = CX[i] * ux + CY[i] * uy;
        feq[i] = WQ[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
    }
}

/* Pseudopotential psi(rho) = rho0 (1 - exp(-rho/rho0)) (Sec. II-A names the
 * pseudopotential model without a formula; this exponential form is the
 * reading used).  Evaluated as -rho0 * expm1(-rho/rho0). */
double orc_psi(double rho, double rho0) { return -rho0 * expm1(-rho / rho0); }

/* Bulk pressure of the pseudopotential fluid with the force below:
 * p = rho c_s^2 + (c_s^2 G / 2) psi^2 = rho/3 + G psi^2 / 6. */
double orc_pressure(double rho, double G, double rho0) {
    double p = orc_psi(rho, rho0);
    return rho / 3.0 + G * p * p / 6.0;
}

/* rho = sum_i f_i, cell by cell (directions summed in order 0..8). */
void orc_density(int nx, int ny, const double* f, double* rho) {
    const long N = (long)nx * ny;
#pragma omp parallel for schedule(static)
    for (long c = 0; c < N; ++c) {
        double s = 0.0;
        for (int i = 0; i < Q; ++i) s += f[i * N + c];
        rho[c] = s;
    }
}

/* Momentum j = sum_i f_i c_i, cell by cell. */
void orc_momentum(int nx, int ny, const double* f, double* jx, double* jy) {
    const long N = (long)nx * ny;
    for (long c = 0; c < N; ++c) {
        double sx = 0.0, sy = 0.0;
        for (int i = 0; i < Q; ++i) {
            sx += f[i * N + c] * CX[i];
            sy += f[i * N + c] * CY[i];
        }
        jx[c] = sx;
        jy[c] = sy;
    }
}

/* Shan-Chen interaction force on a periodic lattice (Sec. II-A: "interaction
 * force between particles"; stencil is the reading used):
 *   F(x) = -G psi(x) sum_{i=1..8} w_i psi(x + c_i) c_i. */
void orc_sc_force(int nx, int ny, const double* psi, double G, double* Fx, double* Fy) {
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            double sx = 0.0, sy = 0.0;
            for (int i = 1; i < Q; ++i) {
                int xn = wrap(x + CX[i], nx), yn = wrap(y + CY[i], ny);
                double pn = psi[(long)yn * nx + xn];
                sx += WQ[i] * pn * CX[i];
                sy += WQ[i] * pn * CY[i];
            }
            long c = (long)y * nx + x;
            Fx[c] = -G * psi[c] * sx;
            Fy[c] = -G * psi[c] * sy;
        }
    }
}

/* BGK collision with the force-shifted equilibrium (Eq. 1, reading: the
 * collision operator is single-relaxation-time BGK, Omega_i = -(f_i - f_i^eq)/tau,
 * and the forcing term enters through the equilibrium velocity
 * u_eq = u + tau F / rho with u = sum_i f_i c_i / rho):
 *   f_i* = f_i - (f_i - f_i^eq(rho, u_eq)) / tau. */
void orc_collide(int nx, int ny, const double* f, const double* Fx, const double* Fy,
                 double tau, double* fpost) {
    const long N = (long)nx * ny;
#pragma omp parallel for schedule(static)
    for (long c = 0; c < N; ++c) {
        double rho = 0.0, jx = 0.0, jy = 0.0;
        for (int i = 0; i < Q; ++i) {
            double fi = f[i * N + c];
            rho += fi;
            jx += fi * CX[i];
            jy += fi * CY[i];
        }
        double ux = jx / rho, uy = jy / rho;
        double uex = ux + tau * Fx[c] / rho;
        double uey = uy + tau * Fy[c] / rho;
        double feq[Q];
        orc_equilibrium(rho, uex, uey, feq);
        for (int i = 0; i < Q; ++i) {
            double fi = f[i * N + c];
            fpost[i * N + c] = fi - (fi - feq[i]) / tau;
        }
    }
}

/* Streaming on a periodic lattice (Eq. 1, left-hand side):
 *   f_i(x + c_i, t+1) = f_i*(x, t). */
void orc_stream(int nx, int ny, const double* fpost, double* fnew) {
    const long N = (long)nx * ny;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            long c = (long)y * nx + x;
            for (int i = 0; i < Q; ++i) {
                long d = (long)wrap(y + CY[i], ny) * nx + wrap(x + CX[i], nx);
                fnew[i * N + d] = fpost[i * N + c];
            }
        }
    }
}

/* n full time steps (Eq. 1): rho -> psi -> F -> collide -> stream, in place on f.
 * Returns 0, or -1 if memory could not be allocated. */
int orc_step(int nx, int ny, double* f, int nsteps, double G, double tau, double rho0) {
    const long N = (long)nx * ny;
    double* rho = (double*)malloc(sizeof(double) * N);
    double* psi = (double*)malloc(sizeof(double) * N);
    double* Fx = (double*)malloc(sizeof(double) * N);
    double* Fy = (double*)malloc(sizeof(double) * N);
    double* fpost = (double*)malloc(sizeof(double) * N * Q);
    if (!rho || !psi || !Fx || !Fy || !fpost) {
        free(rho); free(psi); free(Fx); free(Fy); free(fpost);
        return -1;
    }
    for (int s = 0; s < nsteps; ++s) {
        orc_density(nx, ny, f, rho);
#pragma omp parallel for schedule(static)
        for (long c = 0; c < N; ++c) psi[c] = orc_psi(rho[c], rho0);
        orc_sc_force(nx, ny, psi, G, Fx, Fy);
        orc_collide(nx, ny, f, Fx, Fy, tau, fpost);
        orc_stream(nx, ny, fpost, f);
    }
    free(rho); free(psi); free(Fx); free(Fy); free(fpost);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Initial state (Sec. III-A: droplet in a periodic square box, density ratio
 * and radius given; profile and noise are the readings used):
 *   rho(x) = rho_out + (rho_in - rho_out) * max_k 1/2 (1 - tanh((d_k - R_k)/width))
 *            + noise_amp * (2 U(seed, y*nx + x) - 1),
 * with d_k the periodic minimum-image distance from the cell position (x, y)
 * to the centre of droplet k, U the SplitMix64 uniform above, u = 0 and
 * f_i = f_i^eq(rho, 0) = w_i rho.
 * ------------------------------------------------------------------------- */
static double min_image(double d, double n) {
    double a = fabs(fmod(d, n));
    return a > 0.5 * n ? n - a : a;
}

void orc_init_rho(int nx, int ny, int nd, const double* cx, const double* cy, const double* r,
                  double rho_in, double rho_out, double width, double noise_amp, uint64_t seed,
                  double* rho) {
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            double best = 0.0;
            for (int k = 0; k < nd; ++k) {
                double dx = min_image((double)x - cx[k], (double)nx);
                double dy = min_image((double)y - cy[k], (double)ny);
                double d = sqrt(dx * dx + dy * dy);
                double phi = 0.5 * (1.0 - tanh((d - r[k]) / width));
                if (phi > best) best = phi;
            }
            long c = (long)y * nx + x;
            double u = orc_uniform01(seed, (uint64_t)c);
            rho[c] = rho_out + (rho_in - rho_out) * best + noise_amp * (2.0 * u - 1.0);
        }
    }
}

void orc_init_equilibrium(int nx, int ny, const double* rho, double* f) {
    const long N = (long)nx * ny;
    for (long c = 0; c < N; ++c)
        for (int i = 0; i < Q; ++i) f[i * N + c] = WQ[i] * rho[c];
}

/* ---------------------------------------------------------------------------
 * Metrics (Sec. II-D Eqs. 9-13, discretised in Sec. IV-E Eqs. 14-16).
 * Gradient magnitude by central differences on the periodic lattice with
 * dx = dy = 1 (lattice units):
 *   |grad rho|_{x,y} = sqrt(((rho_{x+1,y} - rho_{x-1,y})/2)^2 + ((rho_{x,y+1} - rho_{x,y-1})/2)^2).
 * ------------------------------------------------------------------------- */
void orc_grad_mag(int nx, int ny, const double* rho, double* g) {
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            double gx = (rho[(long)y * nx + wrap(x + 1, nx)] - rho[(long)y * nx + wrap(x - 1, nx)]) / 2.0;
            double gy = (rho[(long)wrap(y + 1, ny) * nx + x] - rho[(long)wrap(y - 1, ny) * nx + x]) / 2.0;
            g[(long)y * nx + x] = sqrt(gx * gx + gy * gy);
        }
    }
}

/* Metric record, all FP64 (counts as doubles holding integers). */
enum {
    OM_MASS = 0,     /* sum rho                                          */
    OM_W,            /* Eq. 9:  count(|grad rho| > threshold) / N         */
    OM_GMAX,         /* Eq. 10: max |grad rho|                            */
    OM_DRHO,         /* Eq. 11: rho_max - rho_min                         */
    OM_WEFF,         /* Eq. 12/14: sum |grad rho| / (G_max * N), 0 if G_max = 0 */
    OM_EINT,         /* Eq. 13/15: sum |grad rho|^2                        */
    OM_RHOMAX,
    OM_RHOMIN,
    OM_SUMG,
    OM_SUMG2,
    OM_COUNT,
    OM_NFIELDS
};

void orc_metrics_rho(int nx, int ny, const double* rho, double threshold, double* out) {
    const long N = (long)nx * ny;
    double* g = (double*)malloc(sizeof(double) * N);
    orc_grad_mag(nx, ny, rho, g);
    double mass = 0.0, rmax = -INFINITY, rmin = INFINITY, sg = 0.0, sg2 = 0.0, gmax = 0.0;
    long count = 0;
    for (long c = 0; c < N; ++c) {
        mass += rho[c];
        if (rho[c] > rmax) rmax = rho[c];
        if (rho[c] < rmin) rmin = rho[c];
        sg += g[c];
        sg2 += g[c] * g[c];
        if (g[c] > gmax) gmax = g[c];
        if (g[c] > threshold) ++count;
    }
    free(g);
    out[OM_MASS] = mass;
    out[OM_W] = (double)count / (double)N;
    out[OM_GMAX] = gmax;
    out[OM_DRHO] = rmax - rmin;
    out[OM_WEFF] = gmax > 0.0 ? sg / (gmax * (double)N) : 0.0;
    out[OM_EINT] = sg2;
    out[OM_RHOMAX] = rmax;
    out[OM_RHOMIN] = rmin;
    out[OM_SUMG] = sg;
    out[OM_SUMG2] = sg2;
    out[OM_COUNT] = (double)count;
}

/* Laplace measurement for one droplet centred at (cx, cy) (the set-up of
 * Sec. III-A; the estimator is the reading used, the paper has none):
 * starting from rho_in = rho_max and rho_out = rho_min, twice:
 *   R_eq = sqrt(sum(rho - rho_out) / (pi (rho_in - rho_out)))   (equimolar radius)
 *   inner = cells with d < R_eq/2, outer = cells with d > R_eq + 4*width
 *   rho_in, p_in = means over inner; rho_out, p_out = means over outer,
 * with p the bulk pressure above and d the minimum-image distance.
 * out = {R_eq, rho_in, rho_out, p_in, p_out, p_in - p_out}. */
void orc_laplace(int nx, int ny, const double* rho, double cx, double cy, double width, double G,
                 double rho0, double* out) {
    const long N = (long)nx * ny;
    double rin = -INFINITY, rout = INFINITY;
    for (long c = 0; c < N; ++c) {
        if (rho[c] > rin) rin = rho[c];
        if (rho[c] < rout) rout = rho[c];
    }
    double Req = NAN, pin = NAN, pout = NAN;
    for (int it = 0; it < 2; ++it) {
        double excess = 0.0;
        for (long c = 0; c < N; ++c) excess += rho[c] - rout;
        Req = sqrt(excess / (ORC_PI * (rin - rout)));
        double si = 0.0, so = 0.0, spi = 0.0, spo = 0.0;
        long ni = 0, no = 0;
        for (int y = 0; y < ny; ++y) {
            for (int x = 0; x < nx; ++x) {
                double dx = min_image((double)x - cx, (double)nx);
                double dy = min_image((double)y - cy, (double)ny);
                double d = sqrt(dx * dx + dy * dy);
                double r = rho[(long)y * nx + x];
                if (d < 0.5 * Req) {
                    si += r;
                    spi += orc_pressure(r, G, rho0);
                    ++ni;
                }
                if (d > Req + 4.0 * width) {
                    so += r;
                    spo += orc_pressure(r, G, rho0);
                    ++no;
                }
            }
        }
        rin = ni ? si / ni : NAN;
        rout = no ? so / no : NAN;
        pin = ni ? spi / ni : NAN;
        pout = no ? spo / no : NAN;
    }
    out[0] = Req;
    out[1] = rin;
    out[2] = rout;
    out[3] = pin;
    out[4] = pout;
    out[5] = pin - pout;
}

/* ---------------------------------------------------------------------------
 * Network N(x, y) -> (rho, u_x, u_y) (Sec. II-B Eq. 2, Sec. III-B): inputs 2,
 * hidden [64, 128, 128, 64] with tanh, output 3 (linear: the paper lists tanh
 * for the hidden layers only).  Weight blob (float32, row-major W[out][in]):
 *   W1[64 x n_in] b1[64] W2[128x64] b2[128] W3[128x128] b3[128] W4[64x128] b4[64] W5[3x64] b5[3].
 * n_in = 2: the paper's inputs, the cell centre (x^, y^).  n_in = 11: a cell-feature
 * stencil variant (not in the paper): (x^, y^) followed by the density of the cell and
 * of its 8 neighbours, in the velocity order c_0 .. c_8, periodic.
 * mode 0: everything in FP64.
 * mode 1: BF16 emulation of the tensor-core form: h1, h2, h3 (the operands of
 *         layers 2-4) are rounded to BF16 (round to nearest even) after tanh,
 *         W2, W3, W4 are rounded to BF16, products and sums are FP64; layer 1,
 *         h4 and layer 5 stay at full precision.
 * ------------------------------------------------------------------------- */
static const int MLP_HIDDEN[5] = {64, 128, 128, 64, 3};  /* outputs of layers 1..5 */

static int mlp_dim(int n_in, int l) { return l == 0 ? n_in : MLP_HIDDEN[l - 1]; }  /* input width of layer l+1 */

long orc_mlp_blob_size_n(int n_in) {
    long n = 0;
    for (int l = 0; l < 5; ++l) n += (long)MLP_HIDDEN[l] * mlp_dim(n_in, l) + MLP_HIDDEN[l];
    return n;
}

long orc_mlp_blob_size(void) { return orc_mlp_blob_size_n(2); }

/* Seeded weights (Sec. III-B gives the architecture; the configurations call the network
 * "seed-initialised" without a distribution, so the reading used is the common fan-in
 * uniform): entry k of the blob, in blob order (layer by layer, W[out][in] row-major, then
 * b), is (2 U(seed, k) - 1) / sqrt(fan_in) with U the SplitMix64 uniform above and fan_in
 * the input width of its layer, rounded to FP32 (nearest). */
void orc_mlp_init_weights(int n_in, uint64_t seed, float* blob) {
    long k = 0;
    for (int l = 0; l < 5; ++l) {
        int nin = mlp_dim(n_in, l), nout = MLP_HIDDEN[l];
        double bound = 1.0 / sqrt((double)nin);
        long count = (long)nout * nin + nout;
        for (long e = 0; e < count; ++e, ++k) {
            double t = 2.0 * orc_uniform01(seed, (uint64_t)k) - 1.0;
            blob[k] = (float)(t * bound);
        }
    }
}

/* Round a double to the nearest BF16 value (8 significant bits), ties to even. */
double orc_round_bf16(double v) {
    if (v == 0.0 || !isfinite(v)) return v;
    int e;
    double m = frexp(v, &e);          /* v = m * 2^e, 0.5 <= |m| < 1 */
    double s = ldexp(m, 8);           /* 8 significant bits before the point */
    s = nearbyint(s);                 /* default rounding mode: nearest, ties to even */
    return ldexp(s, e - 8);
}

/* Forward pass on n_in inputs `in`; writes the 3 outputs. */
void orc_mlp_forward_n(const float* blob, int mode, int n_in, const double* in, double* out) {
    double a[128], z[128];
    for (int k = 0; k < n_in; ++k) a[k] = in[k];
    const float* p = blob;
    for (int l = 0; l < 5; ++l) {
        int nin = mlp_dim(n_in, l), nout = MLP_HIDDEN[l];
        const float* W = p;
        const float* b = p + (long)nout * nin;
        p = b + nout;
        int tc_layer = (mode == 1) && (l >= 1 && l <= 3); /* layers 2..4 on tensor cores */
        for (int o = 0; o < nout; ++o) {
            double s = 0.0;
            for (int k = 0; k < nin; ++k) {
                double w = (double)W[(long)o * nin + k];
                if (tc_layer) w = orc_round_bf16(w);
                s += w * a[k];
            }
            z[o] = s + (double)b[o];
        }
        if (l < 4) {
            for (int o = 0; o < nout; ++o) {
                double h = tanh(z[o]);
                if (mode == 1 && l <= 2) h = orc_round_bf16(h); /* h1, h2, h3 feed MMA layers */
                a[o] = h;
            }
        } else {
            for (int o = 0; o < nout; ++o) out[o] = z[o];
        }
    }
}

void orc_mlp_forward(const float* blob, int mode, double xh, double yh, double* out) {
    const double in[2] = {xh, yh};
    orc_mlp_forward_n(blob, mode, 2, in, out);
}

/* Network input for cell (x, y): the cell centre mapped to [-1, 1]
 * (the paper says only "x, y coordinates"; the normalisation is the reading used). */
void orc_mlp_inputs(int nx, int ny, int x, int y, double* xh, double* yh) {
    *xh = 2.0 * ((double)x + 0.5) / (double)nx - 1.0;
    *yh = 2.0 * ((double)y + 0.5) / (double)ny - 1.0;
}

/* The n_in inputs of cell (x, y); rho (nx*ny) is read only for n_in = 11. */
void orc_mlp_features(int nx, int ny, const double* rho, int n_in, int x, int y, double* in) {
    orc_mlp_inputs(nx, ny, x, y, &in[0], &in[1]);
    if (n_in == 11) {
        int cx[Q], cy[Q];
        double w[Q];
        orc_lattice_tables(cx, cy, w);
        for (int i = 0; i < Q; ++i) {
            int xn = (x + cx[i] + nx) % nx, yn = (y + cy[i] + ny) % ny;
            in[2 + i] = rho[(long)yn * nx + xn];
        }
    }
}

void orc_mlp_field_n(int nx, int ny, const float* blob, int mode, int n_in, const double* rho, double* out3) {
    const long N = (long)nx * ny;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            double in[11], o[3];
            orc_mlp_features(nx, ny, rho, n_in, x, y, in);
            orc_mlp_forward_n(blob, mode, n_in, in, o);
            long c = (long)y * nx + x;
            out3[c] = o[0];
            out3[N + c] = o[1];
            out3[2 * N + c] = o[2];
        }
    }
}

void orc_mlp_field(int nx, int ny, const float* blob, int mode, double* out3) {
    orc_mlp_field_n(nx, ny, blob, mode, 2, NULL, out3);
}

/* ---------------------------------------------------------------------------
 * Interface correction (Sec. II-C step 3: the network's prediction corrects the
 * lattice state, weighted toward the interface regions; the paper gives no
 * formula, so the operator below is the reading used):
 *   g = |grad rho| (Eq. 16), G_max = max g, m = g / G_max (0 everywhere if G_max = 0)
 *   (rho^, u^) = N(x^, y^)
 *   drho_raw = beta_rho m (rho^ - rho)
 *   drho     = drho_raw - m (sum drho_raw + (M - M0)) / sum m     (total mass -> M0)
 *   rho'     = rho + drho
 *   dj_raw   = beta_u m (rho' u^ - j)          with j = sum_i f_i c_i = rho u
 *   dj       = dj_raw - m sum dj_raw / sum m                      (total momentum kept)
 *   u'       = (j + dj) / rho'
 *   f_i     <- f_i + f_i^eq(rho', u') - f_i^eq(rho, u)            (cells with m > 0 only)
 * Returns 0; -4 if some rho' <= 0 or a corrected quantity is not finite, in
 * which case f is left unchanged.  The network's output field may be supplied
 * precomputed (out3 != NULL, layout of orc_mlp_field) or is evaluated here.
 *
 * Interface band (the correction's emphasis on the interface, Sec. II-C, and the
 * paper's adaptive sampling of interface regions, Sec. IV-D; the band is the reading
 * used): with eps >= 0, cells whose mask m = g / G_max is not above eps count as
 * outside the interface, m = 0 there, so they are neither corrected nor part of the
 * projections, and the network is needed on the band only.  eps = 0 is the
 * correction above (cells with g = 0 already have m = 0).
 * ------------------------------------------------------------------------- */
int orc_correct_eps(int nx, int ny, double* f, const float* blob, int mlp_mode, int n_in, const double* out3_in,
                    double beta_rho, double beta_u, double M0, double eps) {
    const long N = (long)nx * ny;
    double* rho = (double*)malloc(sizeof(double) * N);
    double* jx = (double*)malloc(sizeof(double) * N);
    double* jy = (double*)malloc(sizeof(double) * N);
    double* g = (double*)malloc(sizeof(double) * N);
    double* out3 = (double*)malloc(sizeof(double) * 3 * N);
    double* rhop = (double*)malloc(sizeof(double) * N);
    double* djx = (double*)malloc(sizeof(double) * N);
    double* djy = (double*)malloc(sizeof(double) * N);
    int status = 0;
    orc_density(nx, ny, f, rho);
    orc_momentum(nx, ny, f, jx, jy);
    orc_grad_mag(nx, ny, rho, g);
    if (out3_in)
        memcpy(out3, out3_in, sizeof(double) * 3 * N);
    else
        orc_mlp_field_n(nx, ny, blob, mlp_mode, n_in, rho, out3);  /* the stencil reads this state */

    double gmax = 0.0;
    for (long c = 0; c < N; ++c)
        if (g[c] > gmax) gmax = g[c];
    /* the mask, 0 outside the interface band */
    for (long c = 0; c < N; ++c) {
        double m = gmax > 0.0 ? g[c] / gmax : 0.0;
        g[c] = m > eps ? m : 0.0;
    }
    double sum_m = 0.0, sum_dr = 0.0, M = 0.0;
    for (long c = 0; c < N; ++c) {
        double m = g[c];
        sum_m += m;
        sum_dr += beta_rho * m * (out3[c] - rho[c]);
        M += rho[c];
    }
    if (sum_m > 0.0) {
        double sjx = 0.0, sjy = 0.0;
        for (long c = 0; c < N; ++c) {
            double m = g[c];
            double dr = beta_rho * m * (out3[c] - rho[c]) - m * (sum_dr + (M - M0)) / sum_m;
            rhop[c] = rho[c] + dr;
            djx[c] = beta_u * m * (rhop[c] * out3[N + c] - jx[c]);
            djy[c] = beta_u * m * (rhop[c] * out3[2 * N + c] - jy[c]);
            sjx += djx[c];
            sjy += djy[c];
        }
        for (long c = 0; c < N; ++c) {
            double m = g[c];
            djx[c] -= m * sjx / sum_m;
            djy[c] -= m * sjy / sum_m;
            double upx = (jx[c] + djx[c]) / rhop[c], upy = (jy[c] + djy[c]) / rhop[c];
            if (!(rhop[c] > 0.0) || !isfinite(rhop[c]) || !isfinite(upx) || !isfinite(upy)) status = -4;
        }
        if (status == 0) {
            for (long c = 0; c < N; ++c) {
                double m = g[c];
                if (!(m > 0.0)) continue;
                double fe_new[Q], fe_old[Q];
                orc_equilibrium(rhop[c], (jx[c] + djx[c]) / rhop[c], (jy[c] + djy[c]) / rhop[c], fe_new);
                orc_equilibrium(rho[c], jx[c] / rho[c], jy[c] / rho[c], fe_old);
                for (int i = 0; i < Q; ++i) f[i * N + c] += fe_new[i] - fe_old[i];
            }
        }
    }
    free(rho); free(jx); free(jy); free(g); free(out3); free(rhop); free(djx); free(djy);
    return status;
}

int orc_correct_n(int nx, int ny, double* f, const float* blob, int mlp_mode, int n_in, const double* out3_in,
                  double beta_rho, double beta_u, double M0) {
    return orc_correct_eps(nx, ny, f, blob, mlp_mode, n_in, out3_in, beta_rho, beta_u, M0, 0.0);
}

int orc_correct(int nx, int ny, double* f, const float* blob, int mlp_mode, const double* out3_in,
                double beta_rho, double beta_u, double M0) {
    return orc_correct_n(nx, ny, f, blob, mlp_mode, 2, out3_in, beta_rho, beta_u, M0);
}

/* Total mass sum_c sum_i f_i (cell order, directions 0..8 within a cell). */
double orc_mass(int nx, int ny, const double* f) {
    const long N = (long)nx * ny;
    double M = 0.0;
    for (long c = 0; c < N; ++c) {
        double s = 0.0;
        for (int i = 0; i < Q; ++i) s += f[i * N + c];
        M += s;
    }
    return M;
}

/* ---------------------------------------------------------------------------
 * Coupled run (Sec. II-C with the adaptive intervention frequency of its last
 * paragraph): advance nsteps, and after every step whose count is a multiple
 * of K (K > 0) apply the correction.  Step counts are relative to step0, the
 * lattice's step count on entry.  M0 is the reference mass of the projection.
 * Returns the first nonzero status (the run stops there), else 0.
 * ------------------------------------------------------------------------- */
int orc_run_eps(int nx, int ny, double* f, int nsteps, long step0, int K, double G, double tau,
                double rho0, const float* blob, int mlp_mode, int n_in, double beta_rho, double beta_u, double M0,
                double eps) {
    const long N = (long)nx * ny;
    double* out3 = NULL;
    if (K > 0 && blob && n_in == 2) {
        /* The paper's network depends on coordinates and weights only, so its field
         * is the same at every correction of this run (the stencil variant reads the
         * state and is evaluated at each correction). */
        out3 = (double*)malloc(sizeof(double) * 3 * N);
        orc_mlp_field(nx, ny, blob, mlp_mode, out3);
    }
    int st = 0;
    for (int s = 1; s <= nsteps && st == 0; ++s) {
        st = orc_step(nx, ny, f, 1, G, tau, rho0);
        if (st == 0 && K > 0 && blob && ((step0 + s) % K) == 0)
            st = orc_correct_eps(nx, ny, f, blob, mlp_mode, n_in, out3, beta_rho, beta_u, M0, eps);
    }
    free(out3);
    return st;
}

int orc_run_n(int nx, int ny, double* f, int nsteps, long step0, int K, double G, double tau,
              double rho0, const float* blob, int mlp_mode, int n_in, double beta_rho, double beta_u, double M0) {
    return orc_run_eps(nx, ny, f, nsteps, step0, K, G, tau, rho0, blob, mlp_mode, n_in, beta_rho, beta_u, M0, 0.0);
}

int orc_run(int nx, int ny, double* f, int nsteps, long step0, int K, double G, double tau,
            double rho0, const float* blob, int mlp_mode, double beta_rho, double beta_u, double M0) {
    return orc_run_n(nx, ny, f, nsteps, step0, K, G, tau, rho0, blob, mlp_mode, 2, beta_rho, beta_u, M0);
}
