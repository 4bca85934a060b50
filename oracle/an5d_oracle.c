/*
 * an5d_oracle.c -- plain CPU oracle for iterated star/box Jacobi stencil sweeps.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load this file's library.  The CUDA product
 * path never links, loads or calls it, and shares no code with it.
 *
 * What it computes (AN5D, Section 3.2 "Host Code" and Fig. 5): a
 * double-buffered time loop over the interior of a grid whose boundary
 * (halo) cells are never written.  At every step t each interior point p of
 * the new buffer receives
 *
 *     acc = c[0] * F[p + o_0]                       (one rounded multiply)
 *     acc = fma(c[k], F[p + o_k], acc),  k = 1..n-1  (one rounding each)
 *
 * where F is the old buffer, in the run's precision.  This is the weighted
 * sum of Section 2.1 / Table 4 with the summation order fixed (the paper
 * compiles with fast-math and leaves the order open).  Offsets o_k are
 * listed in the canonical order built by oracle_offsets().
 *
 * Build: cc -O2 -ffp-contract=off -fopenmp -fPIC -shared (no fast-math, no
 * FMA contraction: every multiply, add and fma rounds exactly once as
 * written).  The OpenMP split over the outermost interior axis does not
 * change any result: points are independent within a step (Section 2.2).
 *
 * Arrays are C order, x (last axis) contiguous.  2D grids are (ny, nx),
 * 3D grids (nz, ny, nx); each axis is padded by R cells per side unless the
 * function says "periodic".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define AN5D_STAR 0
#define AN5D_BOX 1

/* ------------------------------------------------------------------------ */
/* Threads                                                                   */

void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Canonical offset order.
 *
 * Star (Table 4, star2d/star3d rows): the centre, then for i = -R..-1, 1..R
 * in that order the axis neighbours (dx=i), (dy=i) and, in 3D, (dz=i).
 * Box (Table 4, box2d/box3d rows; associative partial sums per sub-plane,
 * Section 3.1): the full (2R+1)^d cube with the streaming (slowest) axis
 * outermost: for dz = -R..R, dy = -R..R, dx = -R..R.
 * Writes (dz, dy, dx) triples to off[3k..3k+2]; returns n, or -1 on bad
 * arguments.                                                                */
int oracle_offsets(int ndim, int shape, int R, int32_t *off)
{
    int n = 0;
    if ((ndim != 2 && ndim != 3) || R < 1 || R > 8) return -1;
    if (shape == AN5D_STAR) {
        off[0] = 0; off[1] = 0; off[2] = 0;
        n = 1;
        for (int i = -R; i <= R; ++i) {
            if (i == 0) continue;
            off[3 * n + 0] = 0; off[3 * n + 1] = 0; off[3 * n + 2] = i; ++n;  /* dx = i */
            off[3 * n + 0] = 0; off[3 * n + 1] = i; off[3 * n + 2] = 0; ++n;  /* dy = i */
            if (ndim == 3) {
                off[3 * n + 0] = i; off[3 * n + 1] = 0; off[3 * n + 2] = 0; ++n;  /* dz = i */
            }
        }
        return n;
    }
    if (shape == AN5D_BOX) {
        int zr = (ndim == 3) ? R : 0;
        for (int dz = -zr; dz <= zr; ++dz)
            for (int dy = -R; dy <= R; ++dy)
                for (int dx = -R; dx <= R; ++dx) {
                    off[3 * n + 0] = dz; off[3 * n + 1] = dy; off[3 * n + 2] = dx; ++n;
                }
        return n;
    }
    return -1;
}

/* ------------------------------------------------------------------------ */
/* Geometry of a padded grid (Section 3.1: interior I_Si, halo of width R).  */

typedef struct {
    int64_t nz, ny, nx;     /* interior extents (nz = 1 in 2D) */
    int64_t pz;             /* halo width along z (R in 3D, 0 in 2D) */
    int64_t R;
    int64_t Py, Px;         /* padded extents along y and x */
    int64_t sy, sz;         /* element strides of y and z */
    int64_t total;          /* elements of the padded array */
    int n;
    int64_t lin[1024];      /* linearised offsets, canonical order */
} geom_t;

static int geom_init(geom_t *g, int ndim, int shape, int R, const int64_t *dims,
                     int periodic)
{
    int32_t off[3 * 1024];
    g->n = oracle_offsets(ndim, shape, R, off);
    if (g->n < 0 || g->n > 1024) return -1;
    int64_t h = periodic ? 0 : R;
    g->R = R;
    if (ndim == 2) { g->nz = 1; g->ny = dims[0]; g->nx = dims[1]; g->pz = 0; }
    else { g->nz = dims[0]; g->ny = dims[1]; g->nx = dims[2]; g->pz = h; }
    g->Py = g->ny + 2 * h;
    g->Px = g->nx + 2 * h;
    g->sy = g->Px;
    g->sz = g->Py * g->Px;
    g->total = (g->nz + 2 * g->pz) * g->sz;
    for (int k = 0; k < g->n; ++k)
        g->lin[k] = off[3 * k] * g->sz + off[3 * k + 1] * g->sy + off[3 * k + 2];
    return 0;
}

/* ------------------------------------------------------------------------ */
/* FP32 plain method.                                                        */

static float chain_f32(const float *F, int64_t p, const float *c, const geom_t *g)
{
    float acc = c[0] * F[p + g->lin[0]];
    for (int k = 1; k < g->n; ++k) acc = fmaf(c[k], F[p + g->lin[k]], acc);
    return acc;
}

int oracle_run_f32(int ndim, int shape, int R, const float *c, const int64_t *dims,
                   const float *in, float *out, int64_t T)
{
    geom_t g;
    if (geom_init(&g, ndim, shape, R, dims, 0) || T < 0) return -1;
    float *A = (float *)malloc(sizeof(float) * g.total);
    float *B = (float *)malloc(sizeof(float) * g.total);
    if (!A || !B) { free(A); free(B); return -5; }
    memcpy(A, in, sizeof(float) * g.total);
    memcpy(B, in, sizeof(float) * g.total);   /* halo identical in both buffers */
    for (int64_t t = 0; t < T; ++t) {
        #pragma omp parallel for schedule(static)
        for (int64_t zy = 0; zy < g.nz * g.ny; ++zy) {
            int64_t z = zy / g.ny + g.pz, y = zy % g.ny + g.R;
            int64_t row = z * g.sz + y * g.sy;
            for (int64_t x = g.R; x < g.R + g.nx; ++x)
                B[row + x] = chain_f32(A, row + x, c, &g);
        }
        float *tmp = A; A = B; B = tmp;
    }
    memcpy(out, A, sizeof(float) * g.total);
    free(A); free(B);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* FP64 plain method (also the reference for the precision forms, with the
 * run's rounded coefficients widened to double).                            */

static double chain_f64(const double *F, int64_t p, const double *c, const geom_t *g)
{
    double acc = c[0] * F[p + g->lin[0]];
    for (int k = 1; k < g->n; ++k) acc = fma(c[k], F[p + g->lin[k]], acc);
    return acc;
}

int oracle_run_f64(int ndim, int shape, int R, const double *c, const int64_t *dims,
                   const double *in, double *out, int64_t T)
{
    geom_t g;
    if (geom_init(&g, ndim, shape, R, dims, 0) || T < 0) return -1;
    double *A = (double *)malloc(sizeof(double) * g.total);
    double *B = (double *)malloc(sizeof(double) * g.total);
    if (!A || !B) { free(A); free(B); return -5; }
    memcpy(A, in, sizeof(double) * g.total);
    memcpy(B, in, sizeof(double) * g.total);
    for (int64_t t = 0; t < T; ++t) {
        #pragma omp parallel for schedule(static)
        for (int64_t zy = 0; zy < g.nz * g.ny; ++zy) {
            int64_t z = zy / g.ny + g.pz, y = zy % g.ny + g.R;
            int64_t row = z * g.sz + y * g.sy;
            for (int64_t x = g.R; x < g.R + g.nx; ++x)
                B[row + x] = chain_f64(A, row + x, c, &g);
        }
        double *tmp = A; A = B; B = tmp;
    }
    memcpy(out, A, sizeof(double) * g.total);
    free(A); free(B);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Division-type stencils (Table 4: j2d5pt, j2d9pt, j2d9pt-gol, j3d27pt): the
 * weighted sum of a star or box stencil divided by a constant d at every
 * step.  post = 1 divides (one IEEE division, correctly rounded); post = 2
 * multiplies by r = 1/d, itself rounded once to the run's precision (the
 * paper's remedy for slow division, Section 6, replaces "/N" by "*(1/N)").
 * The two generally differ in the last bit.  The division or multiplication
 * follows the complete chain of the point (the chain is the same as the
 * plain method's).                                                          */

int oracle_run_div_f32(int ndim, int shape, int R, const float *c, float d, int post,
                       const int64_t *dims, const float *in, float *out, int64_t T)
{
    geom_t g;
    if (geom_init(&g, ndim, shape, R, dims, 0) || T < 0 || (post != 1 && post != 2)) return -1;
    const float r = 1.0f / d;
    float *A = (float *)malloc(sizeof(float) * g.total);
    float *B = (float *)malloc(sizeof(float) * g.total);
    if (!A || !B) { free(A); free(B); return -5; }
    memcpy(A, in, sizeof(float) * g.total);
    memcpy(B, in, sizeof(float) * g.total);
    for (int64_t t = 0; t < T; ++t) {
        #pragma omp parallel for schedule(static)
        for (int64_t zy = 0; zy < g.nz * g.ny; ++zy) {
            int64_t z = zy / g.ny + g.pz, y = zy % g.ny + g.R;
            int64_t row = z * g.sz + y * g.sy;
            for (int64_t x = g.R; x < g.R + g.nx; ++x) {
                const float s = chain_f32(A, row + x, c, &g);
                B[row + x] = (post == 1) ? s / d : s * r;
            }
        }
        float *tmp = A; A = B; B = tmp;
    }
    memcpy(out, A, sizeof(float) * g.total);
    free(A); free(B);
    return 0;
}

int oracle_run_div_f64(int ndim, int shape, int R, const double *c, double d, int post,
                       const int64_t *dims, const double *in, double *out, int64_t T)
{
    geom_t g;
    if (geom_init(&g, ndim, shape, R, dims, 0) || T < 0 || (post != 1 && post != 2)) return -1;
    const double r = 1.0 / d;
    double *A = (double *)malloc(sizeof(double) * g.total);
    double *B = (double *)malloc(sizeof(double) * g.total);
    if (!A || !B) { free(A); free(B); return -5; }
    memcpy(A, in, sizeof(double) * g.total);
    memcpy(B, in, sizeof(double) * g.total);
    for (int64_t t = 0; t < T; ++t) {
        #pragma omp parallel for schedule(static)
        for (int64_t zy = 0; zy < g.nz * g.ny; ++zy) {
            int64_t z = zy / g.ny + g.pz, y = zy % g.ny + g.R;
            int64_t row = z * g.sz + y * g.sy;
            for (int64_t x = g.R; x < g.R + g.nx; ++x) {
                const double s = chain_f64(A, row + x, c, &g);
                B[row + x] = (post == 1) ? s / d : s * r;
            }
        }
        double *tmp = A; A = B; B = tmp;
    }
    memcpy(out, A, sizeof(double) * g.total);
    free(A); free(B);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Periodic FP64 variant: no halo, every index wraps modulo the extent.
 * Used only for the plane-wave eigenvalue check (a Fourier mode of a
 * periodic linear stencil is multiplied by lambda = sum_k c_k e^{i theta.o_k}
 * per step).                                                                */

int oracle_run_periodic_f64(int ndim, int shape, int R, const double *c,
                            const int64_t *dims, const double *in, double *out,
                            int64_t T)
{
    geom_t g;
    int32_t off[3 * 1024];
    if (geom_init(&g, ndim, shape, R, dims, 1) || T < 0) return -1;
    oracle_offsets(ndim, shape, R, off);
    double *A = (double *)malloc(sizeof(double) * g.total);
    double *B = (double *)malloc(sizeof(double) * g.total);
    if (!A || !B) { free(A); free(B); return -5; }
    memcpy(A, in, sizeof(double) * g.total);
    for (int64_t t = 0; t < T; ++t) {
        #pragma omp parallel for schedule(static)
        for (int64_t z = 0; z < g.nz; ++z)
            for (int64_t y = 0; y < g.ny; ++y)
                for (int64_t x = 0; x < g.nx; ++x) {
                    double acc = 0.0;
                    for (int k = 0; k < g.n; ++k) {
                        int64_t zz = ((z + off[3 * k]) % g.nz + g.nz) % g.nz;
                        int64_t yy = ((y + off[3 * k + 1]) % g.ny + g.ny) % g.ny;
                        int64_t xx = ((x + off[3 * k + 2]) % g.nx + g.nx) % g.nx;
                        double f = A[zz * g.sz + yy * g.sy + xx];
                        acc = (k == 0) ? c[0] * f : fma(c[k], f, acc);
                    }
                    B[z * g.sz + y * g.sy + x] = acc;
                }
        double *tmp = A; A = B; B = tmp;
    }
    memcpy(out, A, sizeof(double) * g.total);
    free(A); free(B);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* IEEE 754 binary16 <-> binary32, written from the format definition
 * (1 sign bit, 5 exponent bits with bias 15, 10 fraction bits; subnormal
 * unit 2^-24).  Rounding is to nearest, ties to even.                       */

float oracle_f16_to_f32(uint16_t h)
{
    int sign = (h >> 15) & 1;
    int e = (h >> 10) & 0x1F;
    int m = h & 0x3FF;
    float v;
    if (e == 0) v = ldexpf((float)m, -24);
    else if (e == 31) v = m ? NAN : INFINITY;
    else v = ldexpf((float)(1024 + m), e - 25);
    return sign ? -v : v;
}

uint16_t oracle_f32_to_f16(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    uint32_t sign = (u >> 16) & 0x8000u;
    int32_t exp = (int32_t)((u >> 23) & 0xFF);
    uint32_t man = u & 0x7FFFFFu;
    if (exp == 0xFF)                                  /* inf or NaN */
        return (uint16_t)(sign | 0x7C00u | (man ? (0x200u | (man >> 13)) : 0u));
    int32_t e = exp - 127 + 15;                       /* binary16 biased exponent */
    if (e >= 31) return (uint16_t)(sign | 0x7C00u);   /* >= 2^16: overflows */
    if (e >= 1) {                                     /* normal binary16 range */
        uint32_t h = ((uint32_t)e << 10) | (man >> 13);
        uint32_t rest = man & 0x1FFFu;
        if (rest > 0x1000u || (rest == 0x1000u && (h & 1u))) h += 1;  /* may carry to inf */
        return (uint16_t)(sign | h);
    }
    if (exp == 0) return (uint16_t)sign;              /* < 2^-126: rounds to zero */
    /* binary16 subnormal: value = (man | 2^23) * 2^(exp-150) = q * 2^-24 */
    uint32_t m = man | 0x800000u;
    int32_t s = 126 - exp;                            /* >= 14 here */
    if (s >= 32) return (uint16_t)sign;
    uint32_t q = m >> s;
    uint32_t r = m & ((1u << s) - 1u);
    uint32_t half = 1u << (s - 1);
    if (r > half || (r == half && (q & 1u))) q += 1;
    return (uint16_t)(sign | q);
}

/* FP16 storage, FP32 compute: every level is read from binary16, summed in
 * FP32 with the plain chain and rounded back to binary16.                   */
int oracle_run_f16s(int ndim, int shape, int R, const float *c, const int64_t *dims,
                    const uint16_t *in, uint16_t *out, int64_t T)
{
    geom_t g;
    if (geom_init(&g, ndim, shape, R, dims, 0) || T < 0) return -1;
    uint16_t *A = (uint16_t *)malloc(sizeof(uint16_t) * g.total);
    uint16_t *B = (uint16_t *)malloc(sizeof(uint16_t) * g.total);
    if (!A || !B) { free(A); free(B); return -5; }
    memcpy(A, in, sizeof(uint16_t) * g.total);
    memcpy(B, in, sizeof(uint16_t) * g.total);
    for (int64_t t = 0; t < T; ++t) {
        #pragma omp parallel for schedule(static)
        for (int64_t zy = 0; zy < g.nz * g.ny; ++zy) {
            int64_t z = zy / g.ny + g.pz, y = zy % g.ny + g.R;
            int64_t row = z * g.sz + y * g.sy;
            for (int64_t x = g.R; x < g.R + g.nx; ++x) {
                int64_t p = row + x;
                float acc = c[0] * oracle_f16_to_f32(A[p + g.lin[0]]);
                for (int k = 1; k < g.n; ++k)
                    acc = fmaf(c[k], oracle_f16_to_f32(A[p + g.lin[k]]), acc);
                B[p] = oracle_f32_to_f16(acc);
            }
        }
        uint16_t *tmp = A; A = B; B = tmp;
    }
    memcpy(out, A, sizeof(uint16_t) * g.total);
    free(A); free(B);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Compensated FP32 form: the per-point dot product is evaluated with Dot2
 * of Ogita, Rump and Oishi ("Accurate sum and dot product", SIAM J. Sci.
 * Comput. 26(6), 2005, Algorithm 5.3), using the error-free transformations
 * TwoProduct (via fma) and TwoSum (Knuth), over the canonical order.        */

static float dot2_f32(const float *F, int64_t p, const float *c, const geom_t *g)
{
    float a = c[0], b = F[p + g->lin[0]];
    float ph = a * b;                    /* TwoProduct: high part */
    float s = fmaf(a, b, -ph);           /*             exact low part */
    for (int k = 1; k < g->n; ++k) {
        a = c[k];
        b = F[p + g->lin[k]];
        float h = a * b;
        float r = fmaf(a, b, -h);
        float t = ph + h;                /* TwoSum(ph, h) -> (t, q) */
        float z = t - ph;
        float q = (ph - (t - z)) + (h - z);
        ph = t;
        s = s + (q + r);
    }
    return ph + s;
}

int oracle_run_dot2(int ndim, int shape, int R, const float *c, const int64_t *dims,
                    const float *in, float *out, int64_t T)
{
    geom_t g;
    if (geom_init(&g, ndim, shape, R, dims, 0) || T < 0) return -1;
    float *A = (float *)malloc(sizeof(float) * g.total);
    float *B = (float *)malloc(sizeof(float) * g.total);
    if (!A || !B) { free(A); free(B); return -5; }
    memcpy(A, in, sizeof(float) * g.total);
    memcpy(B, in, sizeof(float) * g.total);
    for (int64_t t = 0; t < T; ++t) {
        #pragma omp parallel for schedule(static)
        for (int64_t zy = 0; zy < g.nz * g.ny; ++zy) {
            int64_t z = zy / g.ny + g.pz, y = zy % g.ny + g.R;
            int64_t row = z * g.sz + y * g.sy;
            for (int64_t x = g.R; x < g.R + g.nx; ++x)
                B[row + x] = dot2_f32(A, row + x, c, &g);
        }
        float *tmp = A; A = B; B = tmp;
    }
    memcpy(out, A, sizeof(float) * g.total);
    free(A); free(B);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* FP64 adjoint of the plain method for the loss
 *     L = 0.5 * sum over interior p of (u_T[p] - target[p])^2.
 * Reverse-mode differentiation of the forward time loop, one step at a
 * time, with every state u_0..u_T kept:
 *     g_T[p]   = u_T[p] - target[p]                       (interior p)
 *     dL/dc_k += sum_{p interior} g_{t+1}[p] * u_t[p + o_k]
 *     g_t[q]   = sum_k c_k * g_{t+1}[q - o_k]   (terms with q - o_k outside
 *                                                the interior are absent)
 * for t = T-1 .. 0.  The halo is boundary data, not a parameter: grad_u0
 * is returned on the interior with a zero halo.                             */

int oracle_adjoint_f64(int ndim, int shape, int R, const double *c, const int64_t *dims,
                       const double *u0, const double *target, int64_t T,
                       double *grad_u0, double *grad_c, double *loss)
{
    geom_t g;
    if (geom_init(&g, ndim, shape, R, dims, 0) || T < 0) return -1;
    double *U = (double *)malloc(sizeof(double) * g.total * (size_t)(T + 1));
    double *G = (double *)calloc((size_t)g.total, sizeof(double));
    double *H = (double *)calloc((size_t)g.total, sizeof(double));
    if (!U || !G || !H) { free(U); free(G); free(H); return -5; }
    memcpy(U, u0, sizeof(double) * g.total);
    for (int64_t t = 0; t < T; ++t) {
        const double *A = U + t * g.total;
        double *B = U + (t + 1) * g.total;
        memcpy(B, A, sizeof(double) * g.total);
        for (int64_t z = g.pz; z < g.pz + g.nz; ++z)
            for (int64_t y = g.R; y < g.R + g.ny; ++y)
                for (int64_t x = g.R; x < g.R + g.nx; ++x) {
                    int64_t p = z * g.sz + y * g.sy + x;
                    B[p] = chain_f64(A, p, c, &g);
                }
    }
    const double *UT = U + T * g.total;
    double l = 0.0;
    for (int64_t z = g.pz; z < g.pz + g.nz; ++z)
        for (int64_t y = g.R; y < g.R + g.ny; ++y)
            for (int64_t x = g.R; x < g.R + g.nx; ++x) {
                int64_t p = z * g.sz + y * g.sy + x;
                double d = UT[p] - target[p];
                l += 0.5 * d * d;
                G[p] = d;
            }
    for (int k = 0; k < g.n; ++k) grad_c[k] = 0.0;
    for (int64_t t = T - 1; t >= 0; --t) {
        const double *Ut = U + t * g.total;
        for (int k = 0; k < g.n; ++k) {
            double s = 0.0;
            for (int64_t z = g.pz; z < g.pz + g.nz; ++z)
                for (int64_t y = g.R; y < g.R + g.ny; ++y)
                    for (int64_t x = g.R; x < g.R + g.nx; ++x) {
                        int64_t p = z * g.sz + y * g.sy + x;
                        s += G[p] * Ut[p + g.lin[k]];
                    }
            grad_c[k] += s;
        }
        memset(H, 0, sizeof(double) * g.total);
        for (int64_t z = g.pz; z < g.pz + g.nz; ++z)
            for (int64_t y = g.R; y < g.R + g.ny; ++y)
                for (int64_t x = g.R; x < g.R + g.nx; ++x) {
                    int64_t q = z * g.sz + y * g.sy + x;
                    double s = 0.0;
                    for (int k = 0; k < g.n; ++k) s += c[k] * G[q - g.lin[k]];  /* G halo is 0 */
                    H[q] = s;
                }
        double *tmp = G; G = H; H = tmp;
    }
    memcpy(grad_u0, G, sizeof(double) * g.total);
    *loss = l;
    free(U); free(G); free(H);
    return 0;
}
