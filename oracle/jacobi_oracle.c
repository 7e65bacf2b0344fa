/*
 * jacobi_oracle.c -- plain, slow, obviously-correct CPU oracle for the
 * overdecomposed 3D 7-point FP64 Jacobi sweep.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or
 * calls this file: only the tests, the package smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code, header, table or
 * helper with the CUDA library; it was written from the method's
 * definition, not from the kernels.
 *
 * What it computes (the paper's Jacobi proxy, Sec. V "jacobi2d": the Jacobi
 * iterative method applied on a block-decomposed grid whose blocks exchange
 * halos every iteration, a fixed iteration count, no convergence check;
 * here in 3D with a 7-point stencil):
 *
 *   u^{t+1}[i,j,k] = (((((u[i-1] + u[i+1]) + u[j-1]) + u[j+1])
 *                      + u[k-1]) + u[k+1]) / 6.0
 *
 * over the NX*NY*NZ interior of a padded array whose one-cell shell holds
 * fixed (Dirichlet) values.  Readings of points the paper leaves open:
 *   - weights: mean of the six face neighbours, centre weight 0;
 *   - summation order: x-, x+, y-, y+, z-, z+ left to right, then one IEEE
 *     division by 6.0 (no reciprocal multiply);
 *   - no FMA contraction (built with -ffp-contract=off), no fast-math;
 *   - the shell lies outside the unknowns; its edges and corners are never
 *     read;
 *   - pure Jacobi with two buffers; iters = 0 returns the initial field;
 *   - output = interior only, x fastest (index x + NX*(y + NY*z)).
 *
 * Initial field: the value of padded global cell L (L = gx + (NX+2)*(gy +
 * (NY+2)*gz), gx in [0,NX+1] ...) is the (L+1)-th output of a SplitMix64
 * stream seeded with `seed` (Steele, Lea & Flood, OOPSLA 2014), top 53 bits
 * scaled by 2^-53, i.e. uniform on [0,1).  init_mode 0: interior 0 and the
 * shell random; init_mode 1: every cell random.  The value depends on the
 * global cell only, so every decomposition starts from the same field.
 *
 * Functions:
 *   oracle_splitmix64      SplitMix64 output number (index+1) for a seed
 *   oracle_uniform         that output as a double in [0,1)
 *   oracle_init_padded     fill the padded global array
 *   oracle_sweep           monolithic sweep (the definition), optional
 *                          OpenMP threads over z-planes (same bits)
 *   oracle_split           balanced split of n cells into p blocks
 *   oracle_sweep_decomposed  per-block padded arrays, explicit face copies
 *                          into the neighbours' ghost layers every step
 *   oracle_point           value of one interior cell after `iters` steps,
 *                          computed on its dependency cone only
 *   oracle2d_*             the same for the 2D 5-point Jacobi (the paper's
 *                          own application): init, sweep, decomposed sweep,
 *                          point
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PIDX(nx, ny, gx, gy, gz) \
    ((int64_t)(gx) + ((int64_t)(nx) + 2) * ((int64_t)(gy) + ((int64_t)(ny) + 2) * (int64_t)(gz)))

/* SplitMix64: state advances by the golden-ratio gamma, output is the
 * state passed through the two xor-shift-multiply rounds and a final
 * xor-shift.  Output number n (n >= 1) for seed s is mix(s + n*gamma). */
uint64_t oracle_splitmix64(uint64_t seed, uint64_t index)
{
    uint64_t z = seed + (index + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double oracle_uniform(uint64_t seed, uint64_t index)
{
    return (double)(oracle_splitmix64(seed, index) >> 11) * (1.0 / 9007199254740992.0);
}

/* Padded global array P[(nz+2)][(ny+2)][(nx+2)]. */
void oracle_init_padded(int64_t nx, int64_t ny, int64_t nz, uint64_t seed,
                        int init_mode, double *P)
{
    for (int64_t gz = 0; gz < nz + 2; ++gz)
        for (int64_t gy = 0; gy < ny + 2; ++gy)
            for (int64_t gx = 0; gx < nx + 2; ++gx) {
                int64_t L = PIDX(nx, ny, gx, gy, gz);
                int shell = gx == 0 || gy == 0 || gz == 0 ||
                            gx == nx + 1 || gy == ny + 1 || gz == nz + 1;
                P[L] = (shell || init_mode == 1) ? oracle_uniform(seed, (uint64_t)L) : 0.0;
            }
}

/* One 7-point value from a padded array with row length sx and plane
 * size sxy (in elements), at linear index c. */
static double stencil(const double *u, int64_t c, int64_t sx, int64_t sxy)
{
    double s = u[c - 1] + u[c + 1];
    s = s + u[c - sx];
    s = s + u[c + sx];
    s = s + u[c - sxy];
    s = s + u[c + sxy];
    return s / 6.0;
}

/* Monolithic Jacobi sweep on the padded global array P (in place: after the
 * call P holds u^iters, shell unchanged).  `threads` > 1 splits z-planes over
 * OpenMP threads; every cell is still the same expression, so the bits do not
 * depend on the thread count. */
int oracle_sweep(int64_t nx, int64_t ny, int64_t nz, double *P, int iters, int threads)
{
    int64_t n = (nx + 2) * (ny + 2) * (nz + 2);
    int64_t sx = nx + 2, sxy = (nx + 2) * (ny + 2);
    double *Q = (double *)malloc((size_t)n * sizeof(double));
    if (!Q) return -1;
    memcpy(Q, P, (size_t)n * sizeof(double));
    double *cur = P, *nxt = Q;
    if (threads < 1) threads = 1;
    for (int t = 0; t < iters; ++t) {
#ifdef _OPENMP
#pragma omp parallel for num_threads(threads) schedule(static)
#endif
        for (int64_t gz = 1; gz <= nz; ++gz)
            for (int64_t gy = 1; gy <= ny; ++gy)
                for (int64_t gx = 1; gx <= nx; ++gx) {
                    int64_t c = PIDX(nx, ny, gx, gy, gz);
                    nxt[c] = stencil(cur, c, sx, sxy);
                }
        double *tmp = cur; cur = nxt; nxt = tmp;
    }
    if (cur != P) memcpy(P, cur, (size_t)n * sizeof(double));
    free(Q);
    return 0;
}

/* Interior of the padded array, x fastest. */
void oracle_interior(int64_t nx, int64_t ny, int64_t nz, const double *P, double *out)
{
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x)
                out[x + nx * (y + ny * z)] = P[PIDX(nx, ny, x + 1, y + 1, z + 1)];
}

/* Balanced split of n cells into p consecutive blocks: the first (n mod p)
 * blocks get ceil(n/p) cells, the rest floor(n/p).  Writes p+1 edges. */
int oracle_split(int64_t n, int p, int64_t *edges)
{
    if (p < 1 || n < p) return -1;
    int64_t q = n / p, r = n % p, at = 0;
    edges[0] = 0;
    for (int b = 0; b < p; ++b) {
        at += q + (b < r ? 1 : 0);
        edges[b + 1] = at;
    }
    return 0;
}

/* A block of the decomposed oracle: padded (bx+2)(by+2)(bz+2), two
 * parities. */
typedef struct {
    int64_t x0, y0, z0, bx, by, bz;
    double *buf[2];
} oblock;

#define BIDX(b, lx, ly, lz) \
    ((int64_t)(lx) + ((b)->bx + 2) * ((int64_t)(ly) + ((b)->by + 2) * (int64_t)(lz)))

/* Decomposed sweep: blocks cut at ex[0..px], ey[0..py], ez[0..pz] (ascending,
 * ex[0] = 0, ex[px] = nx).  Each block keeps its own padded copy; after each
 * block has computed its interior for step t+1, every block copies its new
 * boundary planes into the facing ghost layer of each neighbour in the new
 * buffer (halo exchange, Sec. V "jacobi2d").  Ghost layers on the domain
 * boundary hold the shell and never change.  Reads u^0 from P (padded global),
 * writes u^iters back into P's interior. */
int oracle_sweep_decomposed(int64_t nx, int64_t ny, int64_t nz,
                            int px, int py, int pz,
                            const int64_t *ex, const int64_t *ey, const int64_t *ez,
                            double *P, int iters)
{
    int nb = px * py * pz;
    oblock *B = (oblock *)calloc((size_t)nb, sizeof(oblock));
    if (!B) return -1;
    int rc = 0;
    for (int cz = 0; cz < pz; ++cz)
        for (int cy = 0; cy < py; ++cy)
            for (int cx = 0; cx < px; ++cx) {
                oblock *b = &B[cx + px * (cy + py * cz)];
                b->x0 = ex[cx]; b->bx = ex[cx + 1] - ex[cx];
                b->y0 = ey[cy]; b->by = ey[cy + 1] - ey[cy];
                b->z0 = ez[cz]; b->bz = ez[cz + 1] - ez[cz];
                if (b->bx < 1 || b->by < 1 || b->bz < 1) { rc = -2; goto out; }
                int64_t n = (b->bx + 2) * (b->by + 2) * (b->bz + 2);
                for (int p = 0; p < 2; ++p) {
                    b->buf[p] = (double *)calloc((size_t)n, sizeof(double));
                    if (!b->buf[p]) { rc = -1; goto out; }
                }
                /* interior + six ghost faces from the global field (the
                 * global field at a neighbour's cell equals that neighbour's
                 * initial value, so this is the first halo exchange) */
                for (int p = 0; p < 2; ++p)
                    for (int64_t lz = 0; lz < b->bz + 2; ++lz)
                        for (int64_t ly = 0; ly < b->by + 2; ++ly)
                            for (int64_t lx = 0; lx < b->bx + 2; ++lx) {
                                int edge = (lx == 0 || lx == b->bx + 1) +
                                           (ly == 0 || ly == b->by + 1) +
                                           (lz == 0 || lz == b->bz + 1);
                                if (edge > 1) continue; /* edges/corners: unused */
                                b->buf[p][BIDX(b, lx, ly, lz)] =
                                    P[PIDX(nx, ny, b->x0 + lx, b->y0 + ly, b->z0 + lz)];
                            }
            }

    for (int t = 0; t < iters; ++t) {
        int src = t & 1, dst = src ^ 1;
        /* compute every block's interior */
        for (int c = 0; c < nb; ++c) {
            oblock *b = &B[c];
            int64_t sx = b->bx + 2, sxy = (b->bx + 2) * (b->by + 2);
            for (int64_t lz = 1; lz <= b->bz; ++lz)
                for (int64_t ly = 1; ly <= b->by; ++ly)
                    for (int64_t lx = 1; lx <= b->bx; ++lx) {
                        int64_t i = BIDX(b, lx, ly, lz);
                        b->buf[dst][i] = stencil(b->buf[src], i, sx, sxy);
                    }
        }
        /* halo exchange: each block's new boundary planes into its
         * neighbours' ghost layers of the new buffer */
        for (int cz = 0; cz < pz; ++cz)
            for (int cy = 0; cy < py; ++cy)
                for (int cx = 0; cx < px; ++cx) {
                    oblock *b = &B[cx + px * (cy + py * cz)];
                    if (cx > 0) { /* my x=1 plane -> left neighbour's x=bx+1 ghost */
                        oblock *n = &B[(cx - 1) + px * (cy + py * cz)];
                        for (int64_t lz = 1; lz <= b->bz; ++lz)
                            for (int64_t ly = 1; ly <= b->by; ++ly)
                                n->buf[dst][BIDX(n, n->bx + 1, ly, lz)] = b->buf[dst][BIDX(b, 1, ly, lz)];
                    }
                    if (cx < px - 1) { /* my x=bx plane -> right neighbour's x=0 ghost */
                        oblock *n = &B[(cx + 1) + px * (cy + py * cz)];
                        for (int64_t lz = 1; lz <= b->bz; ++lz)
                            for (int64_t ly = 1; ly <= b->by; ++ly)
                                n->buf[dst][BIDX(n, 0, ly, lz)] = b->buf[dst][BIDX(b, b->bx, ly, lz)];
                    }
                    if (cy > 0) {
                        oblock *n = &B[cx + px * ((cy - 1) + py * cz)];
                        for (int64_t lz = 1; lz <= b->bz; ++lz)
                            for (int64_t lx = 1; lx <= b->bx; ++lx)
                                n->buf[dst][BIDX(n, lx, n->by + 1, lz)] = b->buf[dst][BIDX(b, lx, 1, lz)];
                    }
                    if (cy < py - 1) {
                        oblock *n = &B[cx + px * ((cy + 1) + py * cz)];
                        for (int64_t lz = 1; lz <= b->bz; ++lz)
                            for (int64_t lx = 1; lx <= b->bx; ++lx)
                                n->buf[dst][BIDX(n, lx, 0, lz)] = b->buf[dst][BIDX(b, lx, b->by, lz)];
                    }
                    if (cz > 0) {
                        oblock *n = &B[cx + px * (cy + py * (cz - 1))];
                        for (int64_t ly = 1; ly <= b->by; ++ly)
                            for (int64_t lx = 1; lx <= b->bx; ++lx)
                                n->buf[dst][BIDX(n, lx, ly, n->bz + 1)] = b->buf[dst][BIDX(b, lx, ly, 1)];
                    }
                    if (cz < pz - 1) {
                        oblock *n = &B[cx + px * (cy + py * (cz + 1))];
                        for (int64_t ly = 1; ly <= b->by; ++ly)
                            for (int64_t lx = 1; lx <= b->bx; ++lx)
                                n->buf[dst][BIDX(n, lx, ly, 0)] = b->buf[dst][BIDX(b, lx, ly, b->bz)];
                    }
                }
    }
    /* gather interiors of u^iters */
    for (int c = 0; c < nb; ++c) {
        oblock *b = &B[c];
        int fin = iters & 1;
        for (int64_t lz = 1; lz <= b->bz; ++lz)
            for (int64_t ly = 1; ly <= b->by; ++ly)
                for (int64_t lx = 1; lx <= b->bx; ++lx)
                    P[PIDX(nx, ny, b->x0 + lx, b->y0 + ly, b->z0 + lz)] = b->buf[fin][BIDX(b, lx, ly, lz)];
    }
out:
    for (int c = 0; c < nb; ++c) {
        free(B[c].buf[0]);
        free(B[c].buf[1]);
    }
    free(B);
    return rc;
}

/* Value of interior cell (x,y,z) (0-based) after `iters` Jacobi steps of the
 * field that oracle_init_padded(seed, init_mode) defines.  Only the cells the
 * result depends on are computed: the update that produces u^{t+1} is done
 * on the cube of half-width iters-1-t around the target (a box that contains
 * the 7-point stencil's diamond-shaped cone), clipped to the interior; the
 * shell stays fixed.  Same expression per cell as oracle_sweep, so the result is
 * bit-identical to element (x,y,z) of a full sweep. */
int oracle_point(int64_t nx, int64_t ny, int64_t nz, uint64_t seed, int init_mode,
                 int iters, int64_t x, int64_t y, int64_t z, double *out)
{
    if (x < 0 || y < 0 || z < 0 || x >= nx || y >= ny || z >= nz || iters < 0) return -1;
    int64_t R = iters;
    /* padded-global sub-box [lo, hi] (inclusive) holding every cell read */
    int64_t lo[3], hi[3], n[3], c[3] = {x + 1, y + 1, z + 1}, N[3] = {nx, ny, nz};
    for (int a = 0; a < 3; ++a) {
        lo[a] = c[a] - R < 0 ? 0 : c[a] - R;
        hi[a] = c[a] + R > N[a] + 1 ? N[a] + 1 : c[a] + R;
        n[a] = hi[a] - lo[a] + 1;
    }
    int64_t cnt = n[0] * n[1] * n[2];
    double *U = (double *)malloc((size_t)cnt * sizeof(double));
    double *V = (double *)malloc((size_t)cnt * sizeof(double));
    if (!U || !V) { free(U); free(V); return -1; }
    for (int64_t k = 0; k < n[2]; ++k)
        for (int64_t j = 0; j < n[1]; ++j)
            for (int64_t i = 0; i < n[0]; ++i) {
                int64_t gx = lo[0] + i, gy = lo[1] + j, gz = lo[2] + k;
                int64_t L = PIDX(nx, ny, gx, gy, gz);
                int shell = gx == 0 || gy == 0 || gz == 0 ||
                            gx == nx + 1 || gy == ny + 1 || gz == nz + 1;
                U[i + n[0] * (j + n[1] * k)] =
                    (shell || init_mode == 1) ? oracle_uniform(seed, (uint64_t)L) : 0.0;
            }
    memcpy(V, U, (size_t)cnt * sizeof(double));
    int64_t sx = n[0], sxy = n[0] * n[1];
    for (int t = 0; t < iters; ++t) {
        int64_t r = R - 1 - t; /* radius of cells needed after this step */
        int64_t a0[3], a1[3];
        for (int a = 0; a < 3; ++a) {
            a0[a] = c[a] - r < 1 ? 1 : c[a] - r;          /* interior only */
            a1[a] = c[a] + r > N[a] ? N[a] : c[a] + r;
        }
        for (int64_t gz = a0[2]; gz <= a1[2]; ++gz)
            for (int64_t gy = a0[1]; gy <= a1[1]; ++gy)
                for (int64_t gx = a0[0]; gx <= a1[0]; ++gx) {
                    int64_t i = (gx - lo[0]) + sx * ((gy - lo[1]) + n[1] * (gz - lo[2]));
                    V[i] = stencil(U, i, sx, sxy);
                }
        double *tmp = U; U = V; V = tmp;
    }
    *out = U[(c[0] - lo[0]) + sx * ((c[1] - lo[1]) + n[1] * (c[2] - lo[2]))];
    free(U);
    free(V);
    return 0;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ 2D
 *
 * The paper's own application (Sec. V "jacobi2d"): Jacobi on a 2D grid with a
 * 5-point stencil, the mean of the four edge neighbours, summed x-, x+, y-,
 * y+ left to right, then divided by 4 (exact power-of-two scaling; the IEEE
 * quotient).  Padded array Q[(ny+2)][(nx+2)], shell fixed; initial field: the
 * value of padded cell L = gx + (nx+2)*gy is the same SplitMix64 function
 * of (seed, L) as in 3D. */

#define PIDX2(nx, gx, gy) ((int64_t)(gx) + ((int64_t)(nx) + 2) * (int64_t)(gy))

void oracle2d_init_padded(int64_t nx, int64_t ny, uint64_t seed, int init_mode, double *P)
{
    for (int64_t gy = 0; gy < ny + 2; ++gy)
        for (int64_t gx = 0; gx < nx + 2; ++gx) {
            int64_t L = PIDX2(nx, gx, gy);
            int shell = gx == 0 || gy == 0 || gx == nx + 1 || gy == ny + 1;
            P[L] = (shell || init_mode == 1) ? oracle_uniform(seed, (uint64_t)L) : 0.0;
        }
}

static double stencil2d(const double *u, int64_t c, int64_t sx)
{
    double s = u[c - 1] + u[c + 1];
    s = s + u[c - sx];
    s = s + u[c + sx];
    return s / 4.0;
}

int oracle2d_sweep(int64_t nx, int64_t ny, double *P, int iters, int threads)
{
    int64_t n = (nx + 2) * (ny + 2), sx = nx + 2;
    double *Q = (double *)malloc((size_t)n * sizeof(double));
    if (!Q) return -1;
    memcpy(Q, P, (size_t)n * sizeof(double));
    double *cur = P, *nxt = Q;
    if (threads < 1) threads = 1;
    for (int t = 0; t < iters; ++t) {
#ifdef _OPENMP
#pragma omp parallel for num_threads(threads) schedule(static)
#endif
        for (int64_t gy = 1; gy <= ny; ++gy)
            for (int64_t gx = 1; gx <= nx; ++gx) {
                int64_t c = PIDX2(nx, gx, gy);
                nxt[c] = stencil2d(cur, c, sx);
            }
        double *tmp = cur; cur = nxt; nxt = tmp;
    }
    if (cur != P) memcpy(P, cur, (size_t)n * sizeof(double));
    free(Q);
    return 0;
}

/* Block-decomposed 2D sweep: blocks cut at ex[0..px] x ey[0..py]; each block
 * keeps a padded (bx+2)(by+2) copy per parity and, after computing, copies its
 * new boundary rows/columns into the facing ghost cells of its neighbours. */
int oracle2d_sweep_decomposed(int64_t nx, int64_t ny, int px, int py, const int64_t *ex, const int64_t *ey,
                              double *P, int iters)
{
    int nb = px * py;
    typedef struct { int64_t x0, y0, bx, by; double *buf[2]; } blk;
    blk *B = (blk *)calloc((size_t)nb, sizeof(blk));
    if (!B) return -1;
    int rc = 0;
#define BI2(b, lx, ly) ((int64_t)(lx) + ((b)->bx + 2) * (int64_t)(ly))
    for (int cy = 0; cy < py; ++cy)
        for (int cx = 0; cx < px; ++cx) {
            blk *b = &B[cx + px * cy];
            b->x0 = ex[cx]; b->bx = ex[cx + 1] - ex[cx];
            b->y0 = ey[cy]; b->by = ey[cy + 1] - ey[cy];
            if (b->bx < 1 || b->by < 1) { rc = -2; goto out2; }
            for (int p = 0; p < 2; ++p) {
                b->buf[p] = (double *)calloc((size_t)((b->bx + 2) * (b->by + 2)), sizeof(double));
                if (!b->buf[p]) { rc = -1; goto out2; }
                for (int64_t ly = 0; ly < b->by + 2; ++ly)
                    for (int64_t lx = 0; lx < b->bx + 2; ++lx) {
                        int edge = (lx == 0 || lx == b->bx + 1) + (ly == 0 || ly == b->by + 1);
                        if (edge > 1) continue;
                        b->buf[p][BI2(b, lx, ly)] = P[PIDX2(nx, b->x0 + lx, b->y0 + ly)];
                    }
            }
        }
    for (int t = 0; t < iters; ++t) {
        int src = t & 1, dst = src ^ 1;
        for (int c = 0; c < nb; ++c) {
            blk *b = &B[c];
            for (int64_t ly = 1; ly <= b->by; ++ly)
                for (int64_t lx = 1; lx <= b->bx; ++lx) {
                    int64_t i = BI2(b, lx, ly);
                    b->buf[dst][i] = stencil2d(b->buf[src], i, b->bx + 2);
                }
        }
        for (int cy = 0; cy < py; ++cy)
            for (int cx = 0; cx < px; ++cx) {
                blk *b = &B[cx + px * cy];
                if (cx > 0) {
                    blk *n = &B[(cx - 1) + px * cy];
                    for (int64_t ly = 1; ly <= b->by; ++ly)
                        n->buf[dst][BI2(n, n->bx + 1, ly)] = b->buf[dst][BI2(b, 1, ly)];
                }
                if (cx < px - 1) {
                    blk *n = &B[(cx + 1) + px * cy];
                    for (int64_t ly = 1; ly <= b->by; ++ly)
                        n->buf[dst][BI2(n, 0, ly)] = b->buf[dst][BI2(b, b->bx, ly)];
                }
                if (cy > 0) {
                    blk *n = &B[cx + px * (cy - 1)];
                    for (int64_t lx = 1; lx <= b->bx; ++lx)
                        n->buf[dst][BI2(n, lx, n->by + 1)] = b->buf[dst][BI2(b, lx, 1)];
                }
                if (cy < py - 1) {
                    blk *n = &B[cx + px * (cy + 1)];
                    for (int64_t lx = 1; lx <= b->bx; ++lx)
                        n->buf[dst][BI2(n, lx, 0)] = b->buf[dst][BI2(b, lx, b->by)];
                }
            }
    }
    for (int c = 0; c < nb; ++c) {
        blk *b = &B[c];
        for (int64_t ly = 1; ly <= b->by; ++ly)
            for (int64_t lx = 1; lx <= b->bx; ++lx)
                P[PIDX2(nx, b->x0 + lx, b->y0 + ly)] = b->buf[iters & 1][BI2(b, lx, ly)];
    }
out2:
    for (int c = 0; c < nb; ++c) {
        free(B[c].buf[0]);
        free(B[c].buf[1]);
    }
    free(B);
#undef BI2
    return rc;
}

/* Value of interior cell (x, y) after `iters` steps, on its dependency cone
 * (a square of half-width iters-1-t around the target, clipped). */
int oracle2d_point(int64_t nx, int64_t ny, uint64_t seed, int init_mode, int iters, int64_t x, int64_t y,
                   double *out)
{
    if (x < 0 || y < 0 || x >= nx || y >= ny || iters < 0) return -1;
    int64_t R = iters, c[2] = {x + 1, y + 1}, N[2] = {nx, ny}, lo[2], hi[2], n[2];
    for (int a = 0; a < 2; ++a) {
        lo[a] = c[a] - R < 0 ? 0 : c[a] - R;
        hi[a] = c[a] + R > N[a] + 1 ? N[a] + 1 : c[a] + R;
        n[a] = hi[a] - lo[a] + 1;
    }
    double *U = (double *)malloc((size_t)(n[0] * n[1]) * sizeof(double));
    double *V = (double *)malloc((size_t)(n[0] * n[1]) * sizeof(double));
    if (!U || !V) { free(U); free(V); return -1; }
    for (int64_t j = 0; j < n[1]; ++j)
        for (int64_t i = 0; i < n[0]; ++i) {
            int64_t gx = lo[0] + i, gy = lo[1] + j, L = PIDX2(nx, gx, gy);
            int shell = gx == 0 || gy == 0 || gx == nx + 1 || gy == ny + 1;
            U[i + n[0] * j] = (shell || init_mode == 1) ? oracle_uniform(seed, (uint64_t)L) : 0.0;
        }
    memcpy(V, U, (size_t)(n[0] * n[1]) * sizeof(double));
    for (int t = 0; t < iters; ++t) {
        int64_t r = R - 1 - t, a0[2], a1[2];
        for (int a = 0; a < 2; ++a) {
            a0[a] = c[a] - r < 1 ? 1 : c[a] - r;
            a1[a] = c[a] + r > N[a] ? N[a] : c[a] + r;
        }
        for (int64_t gy = a0[1]; gy <= a1[1]; ++gy)
            for (int64_t gx = a0[0]; gx <= a1[0]; ++gx) {
                int64_t i = (gx - lo[0]) + n[0] * (gy - lo[1]);
                V[i] = stencil2d(U, i, n[0]);
            }
        double *tmp = U; U = V; V = tmp;
    }
    *out = U[(c[0] - lo[0]) + n[0] * (c[1] - lo[1])];
    free(U);
    free(V);
    return 0;
}
