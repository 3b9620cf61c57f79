/*
 * hz_oracle.c -- plain CPU FP64 reference for the 2D Helmholtz problem with PML.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is used by tests/, by the smoke check
 * and by the CPU-baseline leg of bench.py.  The solver library never links,
 * calls or reads it, and it shares no code, header or table with the CUDA path.
 *
 * What it computes (all in complex128):
 *   - the discrete operator H of Appendix A (5-point stencil, PML by the
 *     substitution d/dx -> alpha_x d/dx with alpha = 1/(1 + i sigma/omega) and
 *     sigma(d) = (C/delta)(d/delta)^2, Appendix A), in the form printed there:
 *       (H u)_{p,q} = - alpha_x(p)[alpha_x(p+1/2)(u_{p+1,q}-u_{p,q})
 *                                 - alpha_x(p-1/2)(u_{p,q}-u_{p-1,q})]/h^2
 *                     - alpha_z(q)[alpha_z(q+1/2)(u_{p,q+1}-u_{p,q})
 *                                 - alpha_z(q-1/2)(u_{p,q}-u_{p,q-1})]/h^2
 *                     - omega^2 m_{p,q} u_{p,q}
 *     with homogeneous Dirichlet data beyond the extended grid (Appendix A).
 *     In the interior (alpha = 1) this is the stencil of Appendix A's first
 *     display, with the u_{p,q} factor on the mass term restored.
 *   - u = H^{-1} f by banded Gaussian elimination with partial pivoting, and
 *     the transposed solve H^T x = b from the same factors.
 *
 * Grid ("box"): an interior of nxi x nzi nodes (node numbers 1..nxi, 1..nzi),
 * framed by p PML nodes on every side; node positions x_k = k h, interior
 * interval [0, (nxi+1) h]; PML thickness delta = p h.  The global problem,
 * each layer and each cell of the decomposition are all boxes of this kind
 * (Sections 2-4: local problems carry their own absorbing layers).
 * Arrays are row-major [nzi+2p][nxi+2p] (x fastest).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex zc;

typedef struct {
    int nxi, nzi, p;
    double omega, h, C;
    const double *m; /* (nzi+2p) x (nxi+2p) squared slowness */
} hzo_box;

/* sigma at position k (in units of h, k may be half-integer) for an interior
 * of nint nodes: distance beyond [0, (nint+1)h], quadratic profile. */
static double sigma_at(double k, int nint, int p, double h, double C)
{
    if (p <= 0) return 0.0;
    double x = k * h, Lx = (nint + 1) * h, delta = p * h, d = 0.0;
    if (x < 0.0) d = -x;
    else if (x > Lx) d = x - Lx;
    if (d <= 0.0) return 0.0;
    double r = d / delta;
    return (C / delta) * r * r;
}

static zc alpha_at(double k, int nint, int p, double h, double C, double omega)
{
    double s = sigma_at(k, nint, p, h, C);
    return 1.0 / (1.0 + I * (s / omega));
}

/* alpha on axis (0 = x, 1 = z) at array index i (0-based) plus `half` (0 or +-0.5) */
void hzo_alpha(const hzo_box *b, int axis, int n, const double *pos, double *out_re, double *out_im)
{
    int nint = axis == 0 ? b->nxi : b->nzi;
    for (int t = 0; t < n; t++) {
        /* pos is the array index (possibly +-0.5); node number k = pos - p + 1 */
        zc a = alpha_at(pos[t] - b->p + 1.0, nint, b->p, b->h, b->C, b->omega);
        out_re[t] = creal(a);
        out_im[t] = cimag(a);
    }
}

/* The (at most five) nonzeros of row (iz, ix): returns count, fills flat
 * column indices (grid order iz*NX+ix) and values. */
static int row_entries(const hzo_box *b, int iz, int ix, int *cols, zc *vals)
{
    const int NX = b->nxi + 2 * b->p, NZ = b->nzi + 2 * b->p;
    const double h2 = b->h * b->h;
    const double kx = ix - b->p + 1.0, kz = iz - b->p + 1.0;
    const double C = b->C, w = b->omega, h = b->h;
    const int p = b->p;
    zc axc = alpha_at(kx, b->nxi, p, h, C, w);
    zc axp = alpha_at(kx + 0.5, b->nxi, p, h, C, w);
    zc axm = alpha_at(kx - 0.5, b->nxi, p, h, C, w);
    zc azc = alpha_at(kz, b->nzi, p, h, C, w);
    zc azp = alpha_at(kz + 0.5, b->nzi, p, h, C, w);
    zc azm = alpha_at(kz - 0.5, b->nzi, p, h, C, w);
    int n = 0;
    zc diag = axc * (axp + axm) / h2 + azc * (azp + azm) / h2
              - w * w * b->m[(size_t)iz * NX + ix];
    if (iz > 0)      { cols[n] = (iz - 1) * NX + ix; vals[n++] = -azc * azm / h2; }
    if (ix > 0)      { cols[n] = iz * NX + ix - 1;   vals[n++] = -axc * axm / h2; }
    cols[n] = iz * NX + ix; vals[n++] = diag;
    if (ix < NX - 1) { cols[n] = iz * NX + ix + 1;   vals[n++] = -axc * axp / h2; }
    if (iz < NZ - 1) { cols[n] = (iz + 1) * NX + ix; vals[n++] = -azc * azp / h2; }
    return n;
}

/* Single matrix entry H[row, col] (flat grid indices). */
void hzo_entry(const hzo_box *b, long row, long col, double *re, double *im)
{
    const int NX = b->nxi + 2 * b->p;
    int cols[5];
    zc vals[5];
    int n = row_entries(b, (int)(row / NX), (int)(row % NX), cols, vals);
    zc v = 0.0;
    for (int t = 0; t < n; t++)
        if (cols[t] == col) v = vals[t];
    *re = creal(v);
    *im = cimag(v);
}

/* The five stencil coefficients of every row, as planes of NX*NZ complex
 * values in grid order: plane 0 couples (iz-1, ix), 1 (iz, ix-1), 2 the node
 * itself, 3 (iz, ix+1), 4 (iz+1, ix); zero where the neighbour lies beyond
 * the extended grid (Dirichlet). */
void hzo_stencil(const hzo_box *b, zc *planes)
{
    const int NX = b->nxi + 2 * b->p, NZ = b->nzi + 2 * b->p;
    const long N = (long)NX * NZ;
    memset(planes, 0, sizeof(zc) * 5 * N);
    for (int iz = 0; iz < NZ; iz++)
        for (int ix = 0; ix < NX; ix++) {
            int cols[5];
            zc vals[5];
            const long r = (long)iz * NX + ix;
            int n = row_entries(b, iz, ix, cols, vals);
            for (int t = 0; t < n; t++) {
                const long d = cols[t] - r;
                const int k = d == -NX ? 0 : d == -1 ? 1 : d == 0 ? 2 : d == 1 ? 3 : 4;
                planes[k * N + r] = vals[t];
            }
        }
}

/* out[r] = sum_k H[...] u[r] for nrhs vectors of length NX*NZ (grid order). */
void hzo_apply(const hzo_box *b, int nrhs, const zc *u, zc *out)
{
    const int NX = b->nxi + 2 * b->p, NZ = b->nzi + 2 * b->p;
    const long N = (long)NX * NZ;
    for (int r = 0; r < nrhs; r++) {
        const zc *ur = u + r * N;
        zc *o = out + r * N;
        for (int iz = 0; iz < NZ; iz++)
            for (int ix = 0; ix < NX; ix++) {
                int cols[5];
                zc vals[5];
                int n = row_entries(b, iz, ix, cols, vals);
                zc s = 0.0;
                for (int t = 0; t < n; t++) s += vals[t] * ur[cols[t]];
                o[(long)iz * NX + ix] = s;
            }
    }
}

/* ---------------- banded LU with partial pivoting ---------------- */

typedef struct {
    long n;        /* unknowns */
    int kl, ku;    /* band widths of H */
    int ldab;      /* 2 kl + ku + 1 */
    int xfast;     /* 1: unknown index iz*NX+ix, 0: ix*NZ+iz */
    int NX, NZ;
    zc *ab;        /* band storage, column j at ab + j*ldab, A(i,j) at row kl+ku+i-j */
    long *ipiv;
} hzo_lu;

#define AB(F, i, j) ((F)->ab[(size_t)(j) * (F)->ldab + ((F)->kl + (F)->ku + (i) - (j))])

static long grid_to_unknown(const hzo_lu *F, long g)
{
    if (F->xfast) return g;
    long iz = g / F->NX, ix = g % F->NX;
    return ix * F->NZ + iz;
}

void hzo_free(void *handle)
{
    hzo_lu *F = (hzo_lu *)handle;
    if (!F) return;
    free(F->ab);
    free(F->ipiv);
    free(F);
}

/* Factor H; transposed solves reuse the factors (hzo_solve trans = 1).
 * Returns NULL on allocation failure; *info = 0 on success, j+1 if the j-th
 * pivot column is exactly zero. */
void *hzo_factor_ordered(const hzo_box *b, int order, int *info)
{
    const int NX = b->nxi + 2 * b->p, NZ = b->nzi + 2 * b->p;
    hzo_lu *F = (hzo_lu *)calloc(1, sizeof(hzo_lu));
    if (!F) return NULL;
    F->NX = NX;
    F->NZ = NZ;
    F->n = (long)NX * NZ;
    /* order 0: the smaller band width; 1: x fastest (band NX); 2: z fastest (band NZ) */
    F->xfast = order == 1 ? 1 : (order == 2 ? 0 : NX <= NZ);
    int bw = F->xfast ? NX : NZ;
    F->kl = F->ku = bw;
    F->ldab = 2 * F->kl + F->ku + 1;
    F->ab = (zc *)calloc((size_t)F->ldab * F->n, sizeof(zc));
    F->ipiv = (long *)malloc(sizeof(long) * F->n);
    if (!F->ab || !F->ipiv) { hzo_free(F); return NULL; }
    /* assemble */
    for (int iz = 0; iz < NZ; iz++)
        for (int ix = 0; ix < NX; ix++) {
            int cols[5];
            zc vals[5];
            int n = row_entries(b, iz, ix, cols, vals);
            long i = grid_to_unknown(F, (long)iz * NX + ix);
            for (int t = 0; t < n; t++) {
                long j = grid_to_unknown(F, cols[t]);
                AB(F, i, j) = vals[t];
            }
        }
    /* Gaussian elimination with partial (row) pivoting, column by column */
    const long n = F->n;
    const int kl = F->kl, ku = F->ku;
    long ju = 0;
    *info = 0;
    for (long j = 0; j < n; j++) {
        long km = kl < n - 1 - j ? kl : n - 1 - j;
        long jp = 0;
        double amax = cabs(AB(F, j, j));
        for (long i = 1; i <= km; i++) {
            double a = cabs(AB(F, j + i, j));
            if (a > amax) { amax = a; jp = i; }
        }
        F->ipiv[j] = j + jp;
        if (amax == 0.0) { if (*info == 0) *info = (int)(j + 1); continue; }
        long jmax = j + ku + jp;
        if (jmax > n - 1) jmax = n - 1;
        if (jmax > ju) ju = jmax;
        if (jp != 0)
            for (long c = j; c <= ju; c++) {
                zc t = AB(F, j, c);
                AB(F, j, c) = AB(F, j + jp, c);
                AB(F, j + jp, c) = t;
            }
        zc piv = AB(F, j, j);
        for (long i = 1; i <= km; i++) AB(F, j + i, j) /= piv;
        const zc *lcol = &AB(F, j + 1, j);
        #pragma omp parallel for schedule(static) if (ju - j > 256)
        for (long c = j + 1; c <= ju; c++) {
            zc t = AB(F, j, c);
            if (t != 0.0) {
                zc *dst = &AB(F, j + 1, c);
                for (long i = 0; i < km; i++) dst[i] -= lcol[i] * t;
            }
        }
    }
    return F;
}

void *hzo_factor(const hzo_box *b, int *info)
{
    return hzo_factor_ordered(b, 0, info);
}

/* In-place solve for nrhs right-hand sides in grid order (length NX*NZ each).
 * trans = 0: H x = b;  trans = 1: H^T x = b (plain transpose, no conjugate). */
int hzo_solve(void *handle, int nrhs, zc *bvec, int trans)
{
    hzo_lu *F = (hzo_lu *)handle;
    const long n = F->n;
    const int kl = F->kl, kv = F->kl + F->ku;
    zc *w = (zc *)malloc(sizeof(zc) * n);
    if (!w) return -1;
    for (int r = 0; r < nrhs; r++) {
        zc *b = bvec + (size_t)r * n;
        for (long g = 0; g < n; g++) w[grid_to_unknown(F, g)] = b[g];
        if (!trans) {
            for (long j = 0; j < n - 1; j++) {
                long km = kl < n - 1 - j ? kl : n - 1 - j;
                long l = F->ipiv[j];
                if (l != j) { zc t = w[j]; w[j] = w[l]; w[l] = t; }
                zc t = w[j];
                if (t != 0.0)
                    for (long i = 1; i <= km; i++) w[j + i] -= AB(F, j + i, j) * t;
            }
            for (long j = n - 1; j >= 0; j--) {
                w[j] /= AB(F, j, j);
                zc t = w[j];
                long i0 = j - kv > 0 ? j - kv : 0;
                for (long i = i0; i < j; i++) w[i] -= AB(F, i, j) * t;
            }
        } else {
            for (long j = 0; j < n; j++) {
                zc t = w[j];
                long i0 = j - kv > 0 ? j - kv : 0;
                for (long i = i0; i < j; i++) t -= AB(F, i, j) * w[i];
                w[j] = t / AB(F, j, j);
            }
            for (long j = n - 2; j >= 0; j--) {
                long km = kl < n - 1 - j ? kl : n - 1 - j;
                zc t = w[j];
                for (long i = 1; i <= km; i++) t -= AB(F, j + i, j) * w[j + i];
                w[j] = t;
                long l = F->ipiv[j];
                if (l != j) { zc s = w[j]; w[j] = w[l]; w[l] = s; }
            }
        }
        for (long g = 0; g < n; g++) b[g] = w[grid_to_unknown(F, g)];
    }
    free(w);
    return 0;
}
