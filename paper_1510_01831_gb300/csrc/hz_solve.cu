#include <type_traits>
// Online stage: Alg. matrix_free_solver with the nested inner solver.
//   1. Newton potentials: cell solves (local solves), inner sweeps, samples.
//   2. FGMRES on the polarized traces (eq. integral_polarized) with P^GS
//      (eq. preconditioner_GS): matrix-free M (Alg. applyM generalised to the
//      polarized system), downward / upward sweeps and upward reflections.
//   3. Reconstruction of the volume from the traces.
//   4. FP64 residual of the global system; refinement passes repeat 1-3 on it.
// Every layer Green's integral is applied through eq. (factorization):
//   F (M_f) -> inner block-LU sweeps ((M^l)^{-1}) -> E and S (M_u).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "hz_ctx.cuh"
#include "hz_tc.cuh"

namespace hz {

template <> Ops<double2> &ops<double2>(hz_ctx *c) { return c->o64; }
template <> Ops<float2> &ops<float2>(hz_ctx *c) { return c->o32; }

// max that keeps a NaN (std::max drops it when it comes second)
static inline double nanmax(double a, double b) { return (std::isnan(a) || std::isnan(b)) ? NAN : std::max(a, b); }

// right-hand side of element e of a [points][B] array (no 64-bit division for power-of-two B)
__device__ __forceinline__ int rhs_of(long long e, int B) {
    return (B & (B - 1)) == 0 ? (int)(e & (B - 1)) : (int)(e % B);
}

// point of element e of a [points][B] array
__device__ __forceinline__ long long point_of(long long e, int B) {
    return (B & (B - 1)) == 0 ? (e >> (__ffs(B) - 1)) : e / B;
}
static inline int grid1(long long n, int t = 256) { return (int)std::min<long long>((n + t - 1) / t, 65535LL * 8); }

// ----------------------------------------------------------- kernels ---
__device__ inline double2 pml_alpha_s(double k, int nint, int p, double h, double C, double omega) {
    double x = k * h, Lx = (nint + 1) * h, delta = p * h, d = 0.0;
    if (x < 0.0)
        d = -x;
    else if (x > Lx)
        d = x - Lx;
    double sig = 0.0;
    if (d > 0.0 && p > 0) {
        double r = d / delta;
        sig = (C / delta) * r * r;
    }
    double s = sig / omega, den = 1.0 + s * s;
    return make_double2(1.0 / den, -s / den);
}

// global alpha at nodes (n entries) and half nodes (n+1 entries, index i = position i - 1/2)
__global__ void k_global_alpha(int NX, int NZ, int nxi, int nzi, int p, double h, double C, double omega, double2 *ax,
                               double2 *axh, double2 *az, double2 *azh) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= NX) {
        if (i < NX) ax[i] = pml_alpha_s(i - p + 1.0, nxi, p, h, C, omega);
        axh[i] = pml_alpha_s(i - p + 0.5, nxi, p, h, C, omega);
    }
    if (i <= NZ) {
        if (i < NZ) az[i] = pml_alpha_s(i - p + 1.0, nzi, p, h, C, omega);
        azh[i] = pml_alpha_s(i - p + 0.5, nzi, p, h, C, omega);
    }
}

// f [B][N] (batch outer) -> fs [N][B] = f / (alpha_x alpha_z): the row-scaled
// source.  32 x 32 tiles through shared memory keep both sides coalesced.
__global__ void k_src_in(const double2 *__restrict__ f, double2 *fs, const double2 *__restrict__ Dg, long long N,
                         int B, int scale) {
    __shared__ double2 t[32][33];
    const long long g0 = (long long)blockIdx.x * 32;
    const int b0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int b = b0 + r;
        const long long g = g0 + threadIdx.x;
        if (b < B && g < N) {
            double2 v = f[(long long)b * N + g];
            if (scale) v = v * Dg[g];
            t[r][threadIdx.x] = v;
        }
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const long long g = g0 + r;
        const int b = b0 + threadIdx.x;
        if (b < B && g < N) fs[g * B + b] = t[threadIdx.x][r];
    }
}

// u [N][B] -> out [B][N]
__global__ void k_out(const double2 *__restrict__ u, double2 *out, long long N, int B) {
    __shared__ double2 t[32][33];
    const long long g0 = (long long)blockIdx.x * 32;
    const int b0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const long long g = g0 + r;
        const int b = b0 + threadIdx.x;
        if (b < B && g < N) t[r][threadIdx.x] = u[g * B + b];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int b = b0 + r;
        const long long g = g0 + threadIdx.x;
        if (b < B && g < N) out[(long long)b * N + g] = t[threadIdx.x][r];
    }
}

static void transpose_in(hz_ctx *c, const double2 *f, double2 *fs, long long N, int B, bool scale) {
    dim3 grid((unsigned)((N + 31) / 32), (B + 31) / 32), blk(32, 8);
    k_src_in<<<grid, blk, 0, c->st>>>(f, fs, c->d_ginvD, N, B, scale ? 1 : 0);
    HZ_CU(cudaGetLastError());
    c->nl++;
}
static void transpose_out(hz_ctx *c, const double2 *u, double2 *out, long long N, int B) {
    dim3 grid((unsigned)((N + 31) / 32), (B + 31) / 32), blk(32, 8);
    k_out<<<grid, blk, 0, c->st>>>(u, out, N, B);
    HZ_CU(cudaGetLastError());
    c->nl++;
}

// r = fs - H_s u  (row-scaled operator on the global box, precomputed
// coefficients) and per-RHS partial sums of |alpha_x alpha_z r|^2 =
// |(H u - f)_{Appendix A}|^2 (mode 1: |alpha_x alpha_z fs|^2 only, r untouched)
__global__ void k_residual(const double2 *__restrict__ u, const double2 *__restrict__ fs, double2 *r,
                           const double2 *__restrict__ dg, const double2 *__restrict__ cx,
                           const double2 *__restrict__ cz, const double2 *__restrict__ Dg, int NX, int NZ, int B,
                           double *part, int nchunk, int mode) {
    const int b = blockIdx.y * 32 + threadIdx.x;
    const long long N = (long long)NX * NZ;
    const long long chunk = (N + nchunk - 1) / nchunk;
    const long long g0 = blockIdx.x * chunk, g1 = min(N, g0 + chunk);
    double acc = 0.0;
    if (b < B) {
#pragma unroll 4
        for (long long g = g0 + threadIdx.y; g < g1; g += blockDim.y) {
            const int iz = (int)(g / NX), ix = (int)(g % NX);
            double2 v;
            if (mode == 0) {
                double2 Hu = dg[g] * u[g * B + b];
                if (ix > 0) Hu = Hu + cx[g - 1] * u[(g - 1) * B + b];
                if (ix < NX - 1) Hu = Hu + cx[g] * u[(g + 1) * B + b];
                if (iz > 0) Hu = Hu + cz[g - NX] * u[(g - NX) * B + b];
                if (iz < NZ - 1) Hu = Hu + cz[g] * u[(g + NX) * B + b];
                v = fs[g * B + b] - Hu;
                r[g * B + b] = v;
            } else {
                v = fs[g * B + b];
            }
            acc += cabs2(Dg[g] * v);
        }
    }
    __shared__ double red[8][33];
    red[threadIdx.y][threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.y == 0 && b < B) {
        double s = 0;
        for (int y = 0; y < blockDim.y; y++) s += red[y][threadIdx.x];
        part[(long long)blockIdx.x * B + b] = s;
    }
}

// The same residual and norms for batches that divide 256 (B = 2^lgB): a CTA takes R
// whole grid rows; the elements of a row, point-major with the right-hand side
// innermost, are spread over the CTA's threads so that every load and store is
// coalesced and no division by the row length is needed.  A thread always holds
// the same right-hand side (b = tid mod B), and its partial sum is added to those
// of the other threads of that right-hand side in thread order.
__global__ void __launch_bounds__(256) k_residual_rows(const double2 *__restrict__ u, const double2 *__restrict__ fs,
                                                       double2 *r, const double2 *__restrict__ dg,
                                                       const double2 *__restrict__ cx, const double2 *__restrict__ cz,
                                                       const double2 *__restrict__ Dg, int NX, int NZ, int lgB, int R,
                                                       double *part, int mode) {
    const int tid = threadIdx.x, B = 1 << lgB, rowE = NX << lgB;
    const int z0 = blockIdx.x * R, z1 = min(NZ, z0 + R);
    const long long rs = (long long)rowE;
    double acc = 0.0;
    for (int iz = z0; iz < z1; iz++) {
        const long long gb = (long long)iz * NX, eb = gb << lgB;
#pragma unroll 2
        for (int e = tid; e < rowE; e += 256) {
            const int ix = e >> lgB;
            const long long g = gb + ix, i = eb + e;
            double2 v;
            if (mode == 0) {
                double2 Hu = dg[g] * u[i];
                if (ix > 0) Hu = Hu + cx[g - 1] * u[i - B];
                if (ix < NX - 1) Hu = Hu + cx[g] * u[i + B];
                if (iz > 0) Hu = Hu + cz[g - NX] * u[i - rs];
                if (iz < NZ - 1) Hu = Hu + cz[g] * u[i + rs];
                v = fs[i] - Hu;
                r[i] = v;
            } else {
                v = fs[i];
            }
            acc += cabs2(Dg[g] * v);
        }
    }
    __shared__ double red[256];
    red[tid] = acc;
    __syncthreads();
    if (tid < B) {
        double sum = 0;
        for (int t = tid; t < 256; t += B) sum += red[t];
        part[(long long)blockIdx.x * B + tid] = sum;
    }
}

__global__ void k_global_D(const double2 *__restrict__ ax, const double2 *__restrict__ az, int NX, long long N,
                           double2 *D, double2 *invD) {
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < N; g += (long long)gridDim.x * blockDim.x) {
        D[g] = ax[g % NX] * az[g / NX];
        invD[g] = cdiv(make_double2(1.0, 0.0), D[g]);
    }
}

// interface couplings: gamma per global column, beta per layer row (layer-local PML)
__global__ void k_couplings(const LayerDesc *__restrict__ layers, int L, const double2 *__restrict__ ax, int NX,
                            int p, double h, double C, double omega, double2 *gam, double2 *beta) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const double h2 = h * h;
    if (blockIdx.y == 0) {
        if (i < NX) gam[i] = cdiv(make_double2(-1.0, 0.0), h2 * ax[i]);
        return;
    }
    const LayerDesc &ld = layers[blockIdx.y - 1];
    if (i < ld.nz) {
        double2 az = pml_alpha_s(i - p + 1.0, ld.n, p, h, C, omega);
        beta[ld.zoff + i] = cdiv(make_double2(-1.0, 0.0), h2 * az);
    }
}

__global__ void k_reduce_parts(const double *__restrict__ part, int nchunk, int width, double *out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= width) return;
    double s = 0;
    for (int c = 0; c < nchunk; c++) s += part[(long long)c * width + i];
    out[i] = s;
}

// symmetric-form global source [N][B] -> cell volumes (owned region only)
template <class T2>
__global__ void k_scatter(const CellDesc *__restrict__ cells, const double2 *__restrict__ g, T2 *vol, int NX, int B) {
    const CellDesc &cd = cells[blockIdx.y];
    const long long n = (long long)cd.nx * cd.nz * B;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        long long pt = point_of(e, B);
        int b = rhs_of(e, B);
        int jz = (int)(pt / cd.nx), jx = (int)(pt % cd.nx);
        T2 v = czero<T2>();
        if (jz >= cd.row_lo && jz < cd.row_hi && jx >= cd.own_lo && jx < cd.own_lo + cd.no)
            v = to2(g[((long long)(cd.s + jz) * NX + cd.t + jx) * B + b], T2{});
        vol[cd.vol_off * B + e] = v;
    }
}

// inner right-hand side from the cell Newton potentials: interface j gets the
// potential of cell j at its column node w (a-half) and of cell j+1 at column
// node 1 (b-half)
template <class T2>
__global__ void k_gather_inner(const LayerDesc *__restrict__ layers, const CellDesc *__restrict__ cells,
                               const T2 *__restrict__ vol, T2 *inner, int B, int p) {
    const LayerDesc &ld = layers[blockIdx.y];
    const int nz = ld.nz, J = ld.C - 1;
    const long long n = (long long)J * 2 * nz * B;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        int b = rhs_of(e, B);
        long long q = e / B;
        int m = (int)(q % (2 * nz)), j = (int)(q / (2 * nz));
        T2 v;
        if (m < nz) {
            const CellDesc &ca = cells[ld.cell0 + j];
            v = vol[(ca.vol_off + (long long)m * ca.nx + p + ca.w - 1) * B + b];
        } else {
            const CellDesc &cb = cells[ld.cell0 + j + 1];
            v = vol[(cb.vol_off + (long long)(m - nz) * cb.nx + p) * B + b];
        }
        inner[(ld.inner_off + (long long)(j + 1) * 2 * nz + m) * B + b] = v;
    }
}

// Newton potential samples at local rows (0, 1, n, n+1) of every layer, owned columns:
// out [L][4][NX][B]
template <class T2>
__global__ void k_samples(const CellDesc *__restrict__ cells, const T2 *__restrict__ vol, T2 *out, int NX, int B,
                          int p) {
    const CellDesc &cd = cells[blockIdx.y];
    const long long n = 4LL * cd.no * B;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        int b = rhs_of(e, B);
        long long q = e / B;
        int o = (int)(q % cd.no), rho = (int)(q / cd.no);
        int jz = rho == 0 ? p - 1 : (rho == 1 ? p : (rho == 2 ? p + cd.n - 1 : p + cd.n));
        int jx = cd.own_lo + o;
        out[(((long long)cd.l * 4 + rho) * NX + cd.t + jx) * B + b] = vol[(cd.vol_off + (long long)jz * cd.nx + jx) * B + b];
    }
}

// polarized right-hand side: interface k gets rows n, n+1 of layer k (d-part)
// and rows 0, 1 of layer k+1 (u-part)
template <class T2>
__global__ void k_pol_rhs(const T2 *__restrict__ s, double2 *rhs, int K, int NX, int B) {
    const long long n = (long long)K * 4 * NX * B;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        long long xb = e % ((long long)NX * B);
        long long q = e / ((long long)NX * B);
        int comp = (int)(q % 4), k = (int)(q / 4);
        int l = comp < 2 ? k : k + 1;
        int rho = comp == 0 ? 2 : (comp == 1 ? 3 : (comp == 2 ? 0 : 1));
        rhs[e] = to2(s[((long long)l * 4 + rho) * NX * B + xb], double2{});
    }
}

// Stage the two input sets of M for every layer (columns [0,B): set A, [B,2B): set B):
//   set A (rows n, n+1 out): top = d+u of interface l-1, bottom = u of interface l
//   set B (rows 0, 1 out)  : top = d of interface l-1,   bottom = u+d of interface l
template <class T2>
__global__ void k_stage_M(const T2 *__restrict__ x, T2 *lin, int L, int NX, int B) {
    const long long n = (long long)L * 4 * NX * 2 * B;
    const long long rowsz = (long long)NX * B;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        int col = (int)(e % (2 * B));
        long long q = e / (2 * B);
        int xi = (int)(q % NX);
        q /= NX;
        int rho = (int)(q % 4), l = (int)(q / 4);
        int set = col >= B, b = col - set * B;
        T2 v = czero<T2>();
        if (rho < 2 && l > 0) {
            const T2 *I = x + (long long)(l - 1) * 4 * rowsz + (long long)xi * B + b;
            v = I[rho * rowsz];                           // d_a or d_b
            if (!set) v = v + I[(2 + rho) * rowsz];       // + u
        } else if (rho >= 2 && l < L - 1) {
            const T2 *I = x + (long long)l * 4 * rowsz + (long long)xi * B + b;
            v = I[rho * rowsz];                           // u_a or u_b
            if (set) v = v + I[(rho - 2) * rowsz];        // + d
        }
        lin[e] = v;
    }
}

// y = M x from the sampled layer fields (jump_2, jump_4 for the d-rows,
// jump_3, jump_1 for the u-rows), written in FP64
template <class T2>
__global__ void k_combine_M(const T2 *__restrict__ x, const T2 *__restrict__ lout, double2 *y, int L, int NX, int B) {
    const int K = L - 1;
    const long long rowsz = (long long)NX * B;
    const long long n = (long long)K * 4 * rowsz;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        long long xb = e % rowsz;
        int xi = (int)(xb / B), b = (int)(xb % B);
        long long q = e / rowsz;
        int comp = (int)(q % 4), k = (int)(q / 4);
        const T2 *I = x + (long long)k * 4 * rowsz + xb;
        double2 da = to2(I[0], double2{}), db = to2(I[rowsz], double2{});
        double2 ua = to2(I[2 * rowsz], double2{}), ub = to2(I[3 * rowsz], double2{});
        double2 v;
        if (comp < 2) {  // layer k, set A (columns 0..B), rows n (2), n+1 (3)
            double2 s = to2(lout[(((long long)k * 4 + 2 + comp) * NX + xi) * 2 * B + b], double2{});
            v = comp == 0 ? (da + ua) - s : db - s;
        } else {         // layer k+1, set B (columns B..2B), rows 0, 1
            double2 t = to2(lout[(((long long)(k + 1) * 4 + comp - 2) * NX + xi) * 2 * B + B + b], double2{});
            v = comp == 2 ? ua - t : (ub + db) - t;
        }
        y[e] = v;
    }
}

// w = v_u - L d with L d = [-t0, d_b - t1]: here only the -d_b part (t added by the E/S step)
template <class T2>
__global__ void k_gs_fix(T2 *x, int K, int NX, int B) {
    const long long rowsz = (long long)NX * B;
    const long long n = (long long)K * rowsz;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        long long xb = e % rowsz;
        int k = (int)(e / rowsz);
        T2 *I = x + (long long)k * 4 * rowsz + xb;
        I[3 * rowsz] = I[3 * rowsz] - I[rowsz];
    }
}

// -L d -> L d in the u-part, d-part cleared
template <class T2>
__global__ void k_refl_finish(T2 *x, int K, int NX, int B) {
    const long long rowsz = (long long)NX * B;
    const long long n = (long long)K * rowsz;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        long long xb = e % rowsz;
        int k = (int)(e / rowsz);
        T2 *I = x + (long long)k * 4 * rowsz + xb;
        I[2 * rowsz] = czero<T2>() - I[2 * rowsz];
        I[3 * rowsz] = czero<T2>() - I[3 * rowsz];
        I[0] = czero<T2>();
        I[rowsz] = czero<T2>();
    }
}

// traces of the interfaces: tr[k][a|b] = d + u  ([K][2][NX][B])
template <class T2>
__global__ void k_traces(const double2 *__restrict__ x, T2 *tr, int K, int NX, int B) {
    const long long rowsz = (long long)NX * B;
    const long long n = (long long)K * 2 * rowsz;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        long long xb = e % rowsz;
        long long q = e / rowsz;
        int ab = (int)(q % 2), k = (int)(q / 2);
        const double2 *I = x + (long long)k * 4 * rowsz + xb;
        tr[e] = to2(I[ab * rowsz] + I[(2 + ab) * rowsz], T2{});
    }
}

// Interface traces of a field (the checkpoint of a solve): rows a = last
// interior row of layer k and b = first interior row of layer k+1, full
// extended width.  u: [B][N] (FP64), tr: [B][K][2][NX]
__global__ void k_get_traces(const LayerDesc *__restrict__ layers, const double2 *__restrict__ u, double2 *tr, int K,
                             int NX, long long N, int B, int p) {
    const long long n = (long long)B * K * 2 * NX;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(e % NX);
        long long q = e / NX;
        const int ab = (int)(q % 2);
        q /= 2;
        const int k = (int)(q % K), b = (int)(q / K);
        const int row = ab == 0 ? layers[k].s + p + layers[k].n - 1 : layers[k + 1].s + p;
        tr[e] = u[(long long)b * N + (long long)row * NX + x];
    }
}

// Given traces [B][K][2][NX] into the polarized layout [K][4][NX][B] with the
// whole trace on the down-going components (their sum is what the
// reconstruction uses)
__global__ void k_put_traces(const double2 *__restrict__ tr, double2 *x, int K, int NX, int B) {
    const long long n = (long long)K * 4 * NX * B;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int b = rhs_of(e, B);
        long long q = e / B;
        const int xi = (int)(q % NX);
        q /= NX;
        const int comp = (int)(q % 4), k = (int)(q / 4);
        x[e] = comp < 2 ? tr[(((long long)b * K + k) * 2 + comp) * NX + xi] : make_double2(0.0, 0.0);
    }
}

// reconstruction source of every cell: outer interface forcing on rows
// (0,1,n,n+1) x owned columns from the traces, inner interface forcing on
// columns (0,1,w,w+1) from the inner traces (Appendix C forcing, both levels).
// The volume is cleared beforehand; threads visit only the forced points
// (points on both sets get the same value from two threads).
template <class T2>
__global__ void k_recon_src(const CellDesc *__restrict__ cells, const LayerDesc *__restrict__ layers,
                            const T2 *__restrict__ tr, const T2 *__restrict__ inner, T2 *vol2, int L, int NX, int B,
                            int p, const double2 *__restrict__ ggam, const double2 *__restrict__ lbeta) {
    const CellDesc &cd = cells[blockIdx.y];
    const LayerDesc &ld = layers[cd.l];
    const int nx = cd.nx, nz = cd.nz;
    const long long rowsz = (long long)NX * B;
    const int npts = 4 * cd.no + 4 * nz;
    const int r0 = p - 1, r1 = p, rn = p + cd.n - 1, rn1 = p + cd.n;
    const int c0 = p - 1, c1 = p, cw = p + cd.w - 1, cw1 = p + cd.w;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)npts * B;
         e += (long long)gridDim.x * blockDim.x) {
        const int b = rhs_of(e, B);
        const int q = (int)(e / B);
        int jz, jx;
        if (q < 4 * cd.no) {
            const int rr = q / cd.no;
            jz = rr == 0 ? r0 : (rr == 1 ? r1 : (rr == 2 ? rn : rn1));
            jx = cd.own_lo + q % cd.no;
        } else {
            const int qq = q - 4 * cd.no, cc = qq / nz;
            jz = qq % nz;
            jx = cc == 0 ? c0 : (cc == 1 ? c1 : (cc == 2 ? cw : cw1));
        }
        double2 v = make_double2(0.0, 0.0);
        // outer rows: source row node 0 <- +gamma t(row 1), node 1 <- -gamma t(row 0),
        // node n <- -gamma t(row n+1), node n+1 <- +gamma t(row n)
        if (jx >= cd.own_lo && jx < cd.own_lo + cd.no && (jz == r0 || jz == r1 || jz == rn || jz == rn1)) {
            const double2 gam = ggam[cd.t + jx];  // owned columns: cell-local alpha_x = global alpha_x
            const long long gx = (long long)(cd.t + jx) * B + b;
            double2 s = make_double2(0.0, 0.0);
            if (cd.l > 0) {  // top pair: interface l-1
                const T2 *I = tr + (long long)(cd.l - 1) * 2 * rowsz + gx;
                if (jz == r0) s = s + to2(I[rowsz], double2{});
                if (jz == r1) s = s - to2(I[0], double2{});
            }
            if (cd.l < L - 1) {  // bottom pair: interface l
                const T2 *I = tr + (long long)cd.l * 2 * rowsz + gx;
                if (jz == rn) s = s - to2(I[rowsz], double2{});
                if (jz == rn1) s = s + to2(I[0], double2{});
            }
            v = v + gam * s;
        }
        if (jx == c0 || jx == c1 || jx == cw || jx == cw1) {
            const double2 beta = lbeta[ld.zoff + jz];
            const long long n2 = 2LL * nz;
            const T2 *Il = inner + (ld.inner_off + (long long)cd.c * n2) * B;        // interface c-1 (slot c)
            const T2 *Ir = inner + (ld.inner_off + (long long)(cd.c + 1) * n2) * B;  // interface c (slot c+1)
            double2 s = make_double2(0.0, 0.0);
            if (jx == c0) s = s + to2(Il[((long long)nz + jz) * B + b], double2{});   // + x_{c-1,b}
            if (jx == c1) s = s - to2(Il[(long long)jz * B + b], double2{});          // - x_{c-1,a}
            if (jx == cw) s = s - to2(Ir[((long long)nz + jz) * B + b], double2{});   // - x_{c,b}
            if (jx == cw1) s = s + to2(Ir[(long long)jz * B + b], double2{});         // + x_{c,a}
            v = v + beta * s;
        }
        vol2[(cd.vol_off + (long long)jz * nx + jx) * B + b] = to2(v, T2{});
    }
}

// u += Newton potential + interface response on the owned region of every cell
template <class T2>
__global__ void k_accum_u(const CellDesc *__restrict__ cells, const T2 *__restrict__ vol, const T2 *__restrict__ vol2,
                          double2 *u, int NX, int B) {
    const CellDesc &cd = cells[blockIdx.y];
    const int rows = cd.row_hi - cd.row_lo;
    const long long n = (long long)rows * cd.no * B;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        int b = rhs_of(e, B);
        long long q = e / B;
        int jx = cd.own_lo + (int)(q % cd.no), jz = cd.row_lo + (int)(q / cd.no);
        long long o = (cd.vol_off + (long long)jz * cd.nx + jx) * B + b;
        long long g = ((long long)(cd.s + jz) * NX + cd.t + jx) * B + b;
        u[g] = u[g] + to2(vol[o] + vol2[o], double2{});
    }
}

template <class TA, class TB>
__global__ void k_cast(const TA *__restrict__ a, TB *b, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = to2(a[i], TB{});
}

// ---- FGMRES helpers (FP64) ----
// partial[i][chunk][b] = sum over the chunk of conj(V_i) w
// partial sums over point chunks of h[i][b] = <V_i, w> (conjugate-linear in V):
// block (chunk, 32 RHS, vector i)
__global__ void k_dots(const double2 *__restrict__ V, long long vstride, const double2 *__restrict__ w, long long n,
                       int B, int nchunk, double2 *part) {
    const int i = blockIdx.z;
    // batches that divide 32 put 32 / B points side by side in a warp, so that every lane
    // works; wider batches take 32 right-hand sides per warp
    const bool packed = B < 32 && (32 % B) == 0;
    const int P = packed ? 32 / B : 1;
    const int b = packed ? (int)threadIdx.x % B : blockIdx.y * 32 + threadIdx.x;
    const int p0 = packed ? threadIdx.y * P + threadIdx.x / B : threadIdx.y, ps = blockDim.y * P;
    const long long chunk = (n + nchunk - 1) / nchunk;
    const long long x0 = blockIdx.x * chunk, x1 = min(n, x0 + chunk);
    double2 acc = make_double2(0.0, 0.0);
    if (b < B) {
        const double2 *Vi = V + i * vstride;
#pragma unroll 4
        for (long long x = x0 + p0; x < x1; x += ps) {
            const double2 a = Vi[x * B + b], c = w[x * B + b];
            acc.x += a.x * c.x + a.y * c.y;
            acc.y += a.x * c.y - a.y * c.x;
        }
    }
    __shared__ double2 red[8][33];
    red[threadIdx.y][threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.y == 0 && (int)threadIdx.x < (packed ? B : 32) && b < B) {
        double2 s = make_double2(0.0, 0.0);  // rows, then the lanes of this right-hand side, in order
        for (int y = 0; y < blockDim.y; y++)
            for (int l = threadIdx.x; l < 32; l += packed ? B : 32) s = s + red[y][l];
        part[((long long)i * nchunk + blockIdx.x) * B + b] = s;
    }
}

// point chunks of the Arnoldi dot products (blocks = chunks x RHS groups x vectors)
static int dots_chunks(long long n, int B) {
    return (int)std::max<long long>(1, std::min<long long>(n / 64, std::max(64, 512 / ((B + 31) / 32))));
}

// h[i][b] (+)= sum over chunks: one warp per (i, b), lanes over chunks, fixed order
__global__ void k_dots_final(const double2 *__restrict__ part, int nchunk, int B, int nvec, double2 *h, int accum) {
    const int e = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (e >= nvec * B) return;  // uniform over the warp
    const int i = e / B, b = e % B;
    const double2 *p = part + (long long)i * nchunk * B + b;
    double2 s = make_double2(0.0, 0.0);
    for (int c = lane; c < nchunk; c += 32) s = s + p[(long long)c * B];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
        s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
    }
    if (lane == 0) h[e] = accum ? h[e] + s : s;
}

// w -= sum_i V_i h[i]   (coefficients hc[i][b])
__global__ void k_axpy_multi(const double2 *__restrict__ V, long long vstride, const double2 *__restrict__ hc, int nvec,
                             double2 *w, long long n, int B) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n * B; e += (long long)gridDim.x * blockDim.x) {
        int b = rhs_of(e, B);
        double2 s = w[e];
        for (int i = 0; i < nvec; i++) s = s - V[i * vstride + e] * hc[i * B + b];
        w[e] = s;
    }
}

// out = w * scale[b]
__global__ void k_scale(const double2 *__restrict__ w, const double *__restrict__ scale, double2 *out, long long n,
                        int B) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n * B; e += (long long)gridDim.x * blockDim.x)
        out[e] = scale[rhs_of(e, B)] * w[e];
}

// x += sum_j Z_j y[j][b]
template <class T2>
__global__ void k_update_x(const T2 *__restrict__ Z, long long zstride, const double2 *__restrict__ y, int nvec,
                           double2 *x, long long n, int B) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n * B; e += (long long)gridDim.x * blockDim.x) {
        int b = rhs_of(e, B);
        double2 s = x[e];
        for (int j = 0; j < nvec; j++) s = s + to2(Z[j * zstride + e], double2{}) * y[j * B + b];
        x[e] = s;
    }
}

// r = b - w
__global__ void k_sub(const double2 *__restrict__ a, const double2 *__restrict__ w, double2 *r, long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        r[e] = a[e] - w[e];
}

// Bi-CGstab vector updates with per-RHS complex coefficients
// p = r + beta[b] (p - omega[b] v)
__global__ void k_bicg_p(double2 *p, const double2 *__restrict__ r, const double2 *__restrict__ v,
                         const double2 *__restrict__ beta, const double2 *__restrict__ omega, long long n, int B) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n * B; e += (long long)gridDim.x * blockDim.x) {
        const int b = rhs_of(e, B);
        p[e] = r[e] + beta[b] * (p[e] - omega[b] * v[e]);
    }
}
// out = a + coef[b] x
__global__ void k_zaxpy(double2 *out, const double2 *__restrict__ a, const double2 *__restrict__ x,
                        const double2 *__restrict__ coef, long long n, int B) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n * B; e += (long long)gridDim.x * blockDim.x)
        out[e] = a[e] + coef[rhs_of(e, B)] * x[e];
}

// ---------------------------------------- compressed-block LU recursion ---
// The inner block-LU sweeps of a layer with its factors in low-rank form
// (P_j ~ QP_j BP_j, V_j ~ QV_j BV_j, rank r).  With ac_j = [a_{j+1}; c_{j-1}] =
// [BP_{j+1} h_j; BV_{j-1} h_j] computed beforehand (h_j = W_j g_j):
//   forward step j = 1..J-1:  [t_{j+1}; u_j] = ac_j + [M_{j+1}; R_{j-1}] t_j,
//                             t_1 = a_1 (M_{j+1} = BP_{j+1} QP_j, R_{j-1} = BV_{j-1} QP_j),
//   backward step j = J-2..1: s_{j-1} = u_j + N_{j-1} s_j, s_{J-2} = u_{J-1}
//                             (N_{j-1} = BV_{j-1} QV_j),
// and x_j = h_j + QP_j t_j + QV_j s_j follows as one batched product.  One CTA
// per (layer, NB right-hand sides) holds all ac_j in shared memory (u_j replaces
// c_{j-1} once step j has used it), so each step is one product of a matrix
// from the ring with the previous step's vector, and two barriers.  The
// matrices stream in step order through the ring by bulk copies issued ST steps
// ahead (mbarrier-completed, bounded waits); ts_j = [t_j; s_j] (t_0 = 0,
// s_{J-1} = 0) go to global memory for the x_j product.
template <class T2, int NB>
__global__ void __launch_bounds__(256) k_lr_chain(const LayerDesc *__restrict__ layers, const int *__restrict__ ids,
                                                  const T2 *__restrict__ MRN, const T2 *__restrict__ AC, T2 *TS, int r,
                                                  int Bw, int *err) {
    constexpr int ST = 3;                  // ring stages
    constexpr int PT = 2 * 64 * NB / 256;  // outputs per thread for r <= 64
    extern __shared__ __align__(16) unsigned char lsm[];
    __shared__ __align__(8) unsigned long long full[ST];
    __shared__ int s_dead;
    const long long r2 = (long long)r * r;
    const LayerDesc ld = layers[ids[blockIdx.y]];
    const int J = ld.C - 1, n0 = blockIdx.x * NB, tid = threadIdx.x;
    T2 *ring = reinterpret_cast<T2 *>(lsm);  // ST stages of 2 r^2
    T2 *vb0 = ring + ST * 2 * r2;             // the recursion's vector, double-buffered (r x NB)
    T2 *vb1 = vb0 + r * NB;
    T2 *bs = vb1 + r * NB;                    // ac_j, then u_j in rows r..2r-1 ([J][2r][NB])
    const long long vs = 2LL * r * Bw;        // one interface's [2r][Bw] vector in global memory
    const T2 *ac = AC + ld.ac_off * Bw;
    T2 *ts = TS + ld.ac_off * Bw;
    const T2 *mrn = MRN + ld.m_off;
    const int nf = J >= 2 ? J - 1 : 0, nbk = J >= 3 ? J - 2 : 0, ncopy = nf + nbk;
    int q_issued = 0, q_waited = 0;  // thread 0: copies issued / consumed
    auto issue = [&](int q) {  // thread 0: the matrices of step q (forward 2 r^2, backward r^2)
        if (q >= ncopy) return;
        q_issued = q + 1;
        const long long off = q < nf ? (long long)q * 2 * r2 : (long long)nf * 2 * r2 + (long long)(q - nf) * r2;
        const unsigned bytes = (unsigned)((q < nf ? 2 : 1) * r2 * sizeof(T2));
        const unsigned mb = su32(&full[q % ST]);
        mb_expect(mb, bytes);
        bulk_g2s(su32(ring + (q % ST) * 2 * r2), mrn + off, bytes, mb);
    };
    if (tid == 0) {
        for (int i = 0; i < ST; i++) mb_init(su32(&full[i]), 1);
        s_dead = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int q = 0; q < ST; q++) issue(q);
    }
    // all of the layer's ac_j, this CTA's columns; t_0 = 0 and s_{J-1} = 0
    for (int e = tid; e < J * 2 * r * NB; e += 256) {
        const int n = e % NB, row = e / NB;  // row = j * 2r + i
        bs[e] = n0 + n < Bw ? ac[(long long)row * Bw + n0 + n] : czero<T2>();
    }
    for (int e = tid; e < r * NB; e += 256) {
        const int i = e / NB, n = e % NB;
        if (n0 + n < Bw) {
            ts[(long long)i * Bw + n0 + n] = czero<T2>();
            ts[(J - 1) * vs + (long long)(r + i) * Bw + n0 + n] = czero<T2>();
        }
    }
    __syncthreads();
    bool dead = false;
    auto wait = [&](int q) {  // the whole CTA learns a timeout together
        if (tid == 0 && !s_dead) {
            if (!mb_wait(su32(&full[q % ST]), (unsigned)((q / ST) & 1), dead, err))
                s_dead = 1;
            else
                q_waited = q + 1;
        }
        __syncthreads();
        return s_dead == 0;
    };
    // this thread's outputs e = tid + 256 p of one step: out = base + A v, A (m x r, stored
    // transposed) in the ring, v the current vector; rows < r go to vn (the next vector) and to lo (global),
    // rows >= r back into base (u_j) -- each output is read and written by one thread
    auto step = [&](const T2 *A, int m, T2 *base, const T2 *v, T2 *vn, T2 *lo) {
#pragma unroll
        for (int p = 0; p < PT; p++) {
            const int e = tid + 256 * p;
            if (e >= m * NB) continue;
            const int i = e / NB, n = e % NB;
            T2 p0 = base[e], p1 = czero<T2>(), p2 = czero<T2>(), p3 = czero<T2>();
            const T2 *a = A + i;  // the block is stored transposed: element (i, k) at k m + i
            int k = 0;
            for (; k + 3 < r; k += 4) {  // four independent partial sums
                cmac(p0, a[(long long)k * m], v[k * NB + n]);
                cmac(p1, a[(long long)(k + 1) * m], v[(k + 1) * NB + n]);
                cmac(p2, a[(long long)(k + 2) * m], v[(k + 2) * NB + n]);
                cmac(p3, a[(long long)(k + 3) * m], v[(k + 3) * NB + n]);
            }
            for (; k < r; k++) cmac(p0, a[(long long)k * m], v[k * NB + n]);
            const T2 o = (p0 + p1) + (p2 + p3);
            if (i < r) {
                vn[e] = o;
                if (lo && n0 + n < Bw) lo[(long long)i * Bw + n0 + n] = o;
            } else {
                base[e] = o;
            }
        }
        __syncthreads();  // vn complete, v and the ring stage no longer read
    };
    T2 *vc = vb0, *vx = vb1;
    int q = 0;
    if (J >= 2) {
        // t_1 = a_1
        for (int e = tid; e < r * NB; e += 256) {
            const int i = e / NB, n = e % NB;
            vc[e] = bs[e];
            if (n0 + n < Bw) ts[vs + (long long)i * Bw + n0 + n] = bs[e];
        }
        __syncthreads();
        for (int j = 1; j <= J - 1; j++, q++) {  // forward
            if (!wait(q)) break;
            step(ring + (q % ST) * 2 * r2, 2 * r, bs + (long long)j * 2 * r * NB, vc, vx,
                 j + 1 <= J - 1 ? ts + (j + 1) * vs : nullptr);
            if (tid == 0 && !s_dead) issue(q + ST);
            T2 *t = vc;
            vc = vx;
            vx = t;
        }
        if (s_dead == 0) {
            // s_{J-2} = u_{J-1}
            for (int e = tid; e < r * NB; e += 256) {
                const int i = e / NB, n = e % NB;
                const T2 u = bs[(long long)(J - 1) * 2 * r * NB + (r + i) * NB + n];
                vc[e] = u;
                if (n0 + n < Bw) ts[(J - 2) * vs + (long long)(r + i) * Bw + n0 + n] = u;
            }
            __syncthreads();
            for (int j = J - 2; j >= 1; j--, q++) {  // backward: s_{j-1} = u_j + N_{j-1} s_j
                if (!wait(q)) break;
                step(ring + (q % ST) * 2 * r2, r, bs + (long long)j * 2 * r * NB + r * NB, vc, vx,
                     ts + (j - 1) * vs + (long long)r * Bw);
                if (tid == 0 && !s_dead) issue(q + ST);
                T2 *t = vc;
                vc = vx;
                vx = t;
            }
        }
    }
    // after a timeout: let the copies this CTA issued land before it leaves (bounded)
    if (tid == 0 && s_dead) {
        for (int qq = q_waited; qq < q_issued; qq++) mb_wait(su32(&full[qq % ST]), (unsigned)((qq / ST) & 1), dead, err);
    }
    __syncthreads();
}

template <class T2, int NB> static size_t lr_smem(int r, int J) {
    return sizeof(T2) * ((size_t)3 * 2 * r * r + 2 * (size_t)r * NB + (size_t)J * 2 * r * NB);
}

template <class T2, int NB>
static bool lr_chain_cfg(hz_ctx *c, const int *ids, int nl, const T2 *MRN, const T2 *AC, T2 *TS, int Bw) {
    const int r = c->lr_r, J = c->C - 1;
    const size_t sm = lr_smem<T2, NB>(r, J);
    if (sm > 220 * 1024) return false;
    static size_t attr = 0;
    if (sm > 48 * 1024 && sm > attr) {
        HZ_CU(cudaFuncSetAttribute(k_lr_chain<T2, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        attr = sm;
    }
    k_lr_chain<T2, NB><<<dim3((Bw + NB - 1) / NB, nl), 256, sm, c->st>>>(c->d_layers, ids, MRN, AC, TS, r, Bw,
                                                                         c->d_err);
    HZ_CU(cudaGetLastError());
    c->nl++;
    return true;
}

template <class T2>
static void launch_lr_chain(hz_ctx *c, const int *ids, int nl, const T2 *MRN, const T2 *AC, T2 *TS, int Bw) {
    if (c->lr_r > 64) throw HzError(HZ_EINVAL, "compressed-block LU: rank above 64");
    // narrow batches: 4 right-hand sides per CTA (more CTAs, shorter steps); else the
    // widest tile whose vectors fit in shared memory
    bool ok = false;
    if (Bw > 32) ok = lr_chain_cfg<T2, 16>(c, ids, nl, MRN, AC, TS, Bw);
    if (!ok && Bw > 32) ok = lr_chain_cfg<T2, 8>(c, ids, nl, MRN, AC, TS, Bw);
    if (!ok) ok = lr_chain_cfg<T2, 4>(c, ids, nl, MRN, AC, TS, Bw);
    if (!ok) throw HzError(HZ_EINVAL, "compressed-block LU: rank too large for the recursion kernel");
}

// whether the recursion kernel takes a launch of Bw right-hand sides
template <class T2> static bool lr_chain_fits(hz_ctx *c, int Bw) {
    const int r = c->lr_r, J = c->C - 1;
    if (r > 64) return false;
    return lr_smem<T2, 4>(r, J) <= 220 * 1024 || (Bw > 32 && lr_smem<T2, 8>(r, J) <= 220 * 1024);
}

// ------------------------------------------------- problem-list build ---
template <class T2> struct ListBuilder {
    hz_ctx *c;
    Ops<T2> &o;
    std::vector<GemmProb<T2>> v;
    int max_tiles = 0, kmax = 0, max_tiles32 = 0, tc_max_tiles = 0, tc_kchunks = 0, max_m = 0, max_n = 0;
    long long tc_tiles = 0, tiles32 = 0;
    ListBuilder(hz_ctx *c_, Ops<T2> &o_) : c(c_), o(o_) {}

    double bytes = 0, flops = 0;
    // the tensor-core GEMM reads the operators through their TF32 split copies
    void tc_operands(GemmProb<float2> &g) {
        g.Atc = g.A2tc = nullptr;
        if (c->opts.tensor_cores < 2) return;
        g.Atc = tc_split_operator(c, g.A, g.lda, g.M, g.K);
        if (g.K2 > 0) g.A2tc = tc_split_operator(c, g.A2, g.lda2, g.M, g.K2);
    }
    void tc_operands(GemmProb<double2> &) {}
    void push(GemmProb<T2> g) {
        tc_operands(g);
        v.push_back(g);
        max_tiles = std::max(max_tiles, ((g.M + GBM - 1) / GBM) * ((g.N + GBN - 1) / GBN));
        max_tiles32 = std::max(max_tiles32, gemm_tiles(g.M, g.N, 1));
        tiles32 += gemm_tiles(g.M, g.N, 1);
        max_m = std::max(max_m, g.M);
        max_n = std::max(max_n, g.N);
        kmax = std::max(kmax, std::max(g.K, 0) + std::max(g.K2, 0));
        const int tct = ((g.M + GT_M - 1) / GT_M) * ((g.N + GT_N - 1) / GT_N);
        tc_max_tiles = std::max(tc_max_tiles, tct);
        tc_tiles += tct;
        tc_kchunks = std::max(tc_kchunks, (std::max(g.K, 0) + GT_KC - 1) / GT_KC + (std::max(g.K2, 0) + GT_KC - 1) / GT_KC);
        const double es = sizeof(T2);
        const double K = (double)g.K + g.K2;
        bytes += es * ((double)g.M * K + K * g.N + (double)g.M * g.N * (g.beta ? 2 : 1));
        flops += 8.0 * g.M * K * g.N;
    }
    // F-step of layer l: inputs (row q of the layer's 4 trace rows at in[q], global
    // column 0, ld) -> inner right-hand sides (inner buffer with ld ldi, column offset coff)
    void add_F(int l, int mask, const T2 *const in[4], long long ld, int N, T2 *inner, long long ldi, int beta) {
        const LayerDesc &ld_ = c->layers[l];
        const int nz = ld_.nz;
        for (int cc = 0; cc < c->C; cc++) {
            const CellDesc &cd = c->cells[ld_.cell0 + cc];
            const int no = cd.no;
            const long long ocol = (long long)(cd.t + cd.own_lo) * ld;
            for (int t = 0; t < 2; t++) {
                int slot;
                long long roff;
                if (t == 0) {
                    if (cc == 0) continue;
                    slot = cc;        // interface c-1, b-half
                    roff = nz;
                } else {
                    if (cc == c->C - 1) continue;
                    slot = cc + 1;    // interface c, a-half
                    roff = 0;
                }
                GemmProb<T2> g{};
                int q0 = (mask & 1) ? 0 : 2, nq = ((mask & 1) ? 2 : 0) + ((mask & 2) ? 2 : 0);
                g.A = o.F + cd.F_off + (long long)t * nz * 4 * no + (long long)q0 * no;
                g.lda = 4LL * no;
                g.M = nz;
                g.K = nq * no;
                g.N = N;
                g.xseg = no;
                g.ldx = ld;
                for (int q = 0; q < nq; q++) g.X[q] = in[q0 + q] + ocol;
                g.yseg = 1 << 30;
                g.ldy = ldi;
                g.Y[0] = inner + (ld_.inner_off + (long long)slot * 2 * nz + roff) * ldi;
                g.beta = beta;
                g.alpha = 1.f;
                push(g);
            }
        }
    }
    // E (+ S) step of layer l: out rows selected by outmask into out[q] (global col 0, ldo);
    // E reads the inner traces (ld ldi), S the outer inputs (if inmask != 0)
    void add_ES(int l, int inmask, const T2 *const in[4], long long ld, int outmask, T2 *const out[4], long long ldo,
                const T2 *inner, long long ldi, int N, int beta) {
        const LayerDesc &ld_ = c->layers[l];
        const int nz = ld_.nz;
        for (int cc = 0; cc < c->C; cc++) {
            const CellDesc &cd = c->cells[ld_.cell0 + cc];
            const int no = cd.no;
            int r0 = (outmask & 1) ? 0 : 2, nr = ((outmask & 1) ? 2 : 0) + ((outmask & 2) ? 2 : 0);
            GemmProb<T2> g{};
            g.A = o.E + cd.E_off + (long long)r0 * no * 4 * nz;
            g.lda = 4LL * nz;
            g.M = nr * no;
            g.K = 4 * nz;
            g.N = N;
            g.xseg = 1 << 30;
            g.ldx = ldi;
            g.X[0] = inner + (ld_.inner_off + (long long)cd.c * 2 * nz) * ldi;
            g.yseg = no;
            g.ldy = ldo;
            const long long ocol_o = (long long)(cd.t + cd.own_lo) * ldo;
            for (int q = 0; q < nr; q++) g.Y[q] = out[r0 + q] + ocol_o;
            g.beta = beta;
            g.alpha = 1.f;
            if (inmask) {
                int q0 = (inmask & 1) ? 0 : 2, nq = ((inmask & 1) ? 2 : 0) + ((inmask & 2) ? 2 : 0);
                g.A2 = o.S + cd.S_off + (long long)r0 * no * 4 * no + (long long)q0 * no;
                g.lda2 = 4LL * no;
                g.K2 = nq * no;
                g.xseg2 = no;
                g.ldx2 = ld;
                const long long ocol = (long long)(cd.t + cd.own_lo) * ld;
                for (int q = 0; q < nq; q++) g.X2[q] = in[q0 + q] + ocol;
            }
            push(g);
        }
    }
    // a layer's Green's integral through the composites (compressed-block LU): every cell's
    // out rows r0, r0+1 (+)= P2 (trace rows q0 .. q0+nq-1 over the cell's input range) ...
    void add_compP2(int l, int q0, int nq, const T2 *const in[4], long long ld, int r0, T2 *const out[4],
                    long long ldo, int N, int beta) {
        const LayerDesc &ld_ = c->layers[l];
        for (int cc = 0; cc < c->C; cc++) {
            const CellDesc &cd = c->cells[ld_.cell0 + cc];
            const long long gs = cd.t + cd.own_lo - cd.cl;  // first global column of the input range
            GemmProb<T2> g{};
            g.A = o.CP2 + cd.P2_off + (long long)r0 * cd.no * 4 * cd.Lt + (long long)q0 * cd.Lt;
            g.lda = 4LL * cd.Lt;
            g.M = 2 * cd.no;
            g.K = nq * cd.Lt;
            g.N = N;
            g.xseg = cd.Lt;
            g.ldx = ld;
            for (int q = 0; q < nq; q++) g.X[q] = in[q0 + q] + gs * ld;
            g.yseg = cd.no;
            g.ldy = ldo;
            for (int q = 0; q < 2; q++) g.Y[q] = out[r0 + q] + (long long)(cd.t + cd.own_lo) * ldo;
            g.beta = beta;
            g.alpha = 1.f;
            push(g);
        }
    }
    // ... and every interface's ac = P1 (the same rows over its two cells), ac with ld ldac
    void add_compP1(int l, int q0, int nq, const T2 *const in[4], long long ld, T2 *acv, long long ldac, int N) {
        const LayerDesc &ld_ = c->layers[l];
        const int r = c->lr_r;
        for (int cc = 0; cc + 1 < c->C; cc++) {
            const CellDesc &cd = c->cells[ld_.cell0 + cc], &cn = c->cells[ld_.cell0 + cc + 1];
            const int L2 = cd.no + cn.no;
            GemmProb<T2> g{};
            g.A = o.CP1 + cd.P1_off + (long long)q0 * L2;
            g.lda = 4LL * L2;
            g.M = 2 * r;
            g.K = nq * L2;
            g.N = N;
            g.xseg = L2;
            g.ldx = ld;
            for (int q = 0; q < nq; q++) g.X[q] = in[q0 + q] + (long long)(cd.t + cd.own_lo) * ld;
            g.yseg = 1 << 30;
            g.ldy = ldac;
            g.Y[0] = acv + (ld_.ac_off + (long long)cc * 2 * r) * ldac;
            g.beta = 0;
            g.alpha = 1.f;
            push(g);
        }
    }
    void add_compA(int l, int q0, int nq, const T2 *const in[4], long long ld, int r0, T2 *const out[4],
                   long long ldo, T2 *acv, int N) {
        add_compP2(l, q0, nq, in, ld, r0, out, ldo, N, 1);
        add_compP1(l, q0, nq, in, ld, acv, N, N);
    }
    // ... then every cell's out rows r0, r0+1 += P3 [ts of interface c-1; ts of interface c]
    // (ts with ld ldts)
    void add_compC(int l, int r0, T2 *const out[4], long long ldo, const T2 *tsv, long long ldts, int N) {
        const LayerDesc &ld_ = c->layers[l];
        const int r = c->lr_r, C = c->C;
        if (C < 2) return;
        for (int cc = 0; cc < C; cc++) {
            const CellDesc &cd = c->cells[ld_.cell0 + cc];
            GemmProb<T2> g{};
            g.A = o.CP3 + cd.P3_off + (long long)r0 * cd.no * 4 * r;
            g.lda = 4LL * r;
            g.M = 2 * cd.no;
            g.K = (cc == 0 || cc == C - 1) ? 2 * r : 4 * r;
            if (cc == 0) g.A += 2 * r;  // no interface on the left
            g.N = N;
            g.xseg = 1 << 30;
            g.ldx = ldts;
            g.X[0] = tsv + (ld_.ac_off + (long long)std::max(cc - 1, 0) * 2 * r) * ldts;
            g.yseg = cd.no;
            g.ldy = ldo;
            for (int q = 0; q < 2; q++) g.Y[q] = out[r0 + q] + (long long)(cd.t + cd.own_lo) * ldo;
            g.beta = 1;
            g.alpha = 1.f;
            push(g);
        }
    }
    ProbList<T2> finish() {
        if (c->tca_pending) {  // split copies built on this stream are complete before any stream reads them
            HZ_CU(cudaStreamSynchronize(c->st));
            c->tca_pending = false;
        }
        ProbList<T2> pl;
        pl.n = (int)v.size();
        pl.max_tiles = max_tiles;
        pl.kmax = kmax;
        pl.max_tiles32 = max_tiles32;
        pl.tc_max_tiles = tc_max_tiles;
        pl.tc_kchunks = tc_kchunks;
        pl.tc_tiles = tc_tiles;
        pl.tiles32 = tiles32;
        pl.max_m = max_m;
        pl.max_n = max_n;
        pl.bytes = bytes;
        pl.flops = flops;
        bytes = flops = 0;
        if (pl.n) {
            pl.d = (GemmProb<T2> *)c->dalloc(sizeof(GemmProb<T2>) * v.size());
            HZ_CU(cudaMemcpy(pl.d, v.data(), sizeof(GemmProb<T2>) * v.size(), cudaMemcpyHostToDevice));
        }
        v.clear();
        max_tiles = kmax = max_tiles32 = tc_max_tiles = tc_kchunks = max_m = max_n = 0;
        tc_tiles = tiles32 = 0;
        return pl;
    }
};

// K slices per tile: launches with fewer tiles than GEMM_SPLIT_TILES and a
// long K are split so that the whole GPU works on them
static int gemm_split(long long tiles, int kmax) {
    if (tiles >= GEMM_SPLIT_TILES || kmax < 512) return 1;
    const long long s = (GEMM_SPLIT_TILES + tiles - 1) / tiles;
    return (int)std::max(1LL, std::min<long long>({8, s, kmax / 256}));  // >= 256 of K per split
}

// K slices per tile of the tensor-core GEMM: launches with few tiles take as many
// slices as fit one CTA per SM in a single wave, at least 2 chunks of K per slice,
// at most 8, within the workspace
static int gemm_tc_split(const ProbList<float2> &pl) {
    if (pl.tc_tiles * 2 > GEMM_TC_SPLIT_TILES || pl.tc_kchunks < 4) return 1;
    const long long slots = (long long)pl.n * pl.tc_max_tiles;
    const long long s = std::min<long long>({GEMM_TC_SPLIT_TILES / pl.tc_tiles, (long long)pl.tc_kchunks / 2, 8,
                                             GEMM_TC_WS_TILES / std::max(1LL, slots)});
    return (int)std::max(1LL, s);
}

static bool run_tc(hz_ctx *c, const ProbList<float2> &pl) {
    if (c->opts.tensor_cores < 2) return false;
    // small launches (a sweep step's F products: ~30 tiles x 9 chunks) stay on the SIMT
    // kernel, whose fixed cost per launch is lower
    if (pl.tc_tiles * pl.tc_kchunks < GEMM_TC_MIN_WORK) return false;
    const int split = gemm_tc_split(pl);
    if (split > 1 && !c->tcg_ws) {
        c->tcg_ws = (float2 *)c->dalloc(sizeof(float2) * (size_t)GEMM_TC_WS_TILES * GT_M * GT_N);
        c->tcg_cnt = (int *)c->dalloc(sizeof(int) * GEMM_TC_WS_TILES);
        HZ_CU(cudaMemsetAsync(c->tcg_cnt, 0, sizeof(int) * GEMM_TC_WS_TILES, c->st));
    }
    c->kt_begin(2, pl.bytes, pl.flops);
    launch_gemm_tc(pl.d, pl.n, pl.tc_max_tiles, split, c->tcg_ws, c->tcg_cnt, c->d_err, c->st, &c->nl);
    c->kt_end();
    return true;
}
static bool run_tc(hz_ctx *, const ProbList<double2> &) { return false; }

template <class T2> static void run(hz_ctx *c, const ProbList<T2> &pl, int cls = 2) {
    if (!pl.n) return;
    if (run_tc(c, pl)) return;
    // FP32 lists with panels of <= NW_NB columns: the narrow kernel, a stream over the
    // operators with a block in flight per warp during the products of another; lists with
    // few tiles and long K are cut into K slices so that one wave of NW_CTAS_PER_SM CTAs
    // per SM takes part, each warp with at least two blocks
    static const bool narrow = !getenv("HZ_GEMM") || strcmp(getenv("HZ_GEMM"), "tiled") != 0;
    if (sizeof(T2) == 8 && narrow && pl.max_n <= NW_NB) {
        const long long slots = (long long)pl.n * pl.max_tiles32, wave = 152LL * NW_CTAS_PER_SM;
        const int nbk = (pl.kmax + NW_KB - 1) / NW_KB;
        int split = 1;
        if (pl.tiles32 > 0 && slots <= NW_WS_SLOTS)
            split = (int)std::max(1LL, std::min<long long>({8, wave / pl.tiles32, NW_WS_SLOTS / slots,
                                                            std::max(1, nbk / (2 * NW_WPC))}));
        if (split > 1 && !c->nw_ws) {
            c->nw_ws = (float2 *)c->dalloc(sizeof(float2) * (size_t)NW_WS_SLOTS * 32 * NW_NB);
            c->nw_cnt = (int *)c->dalloc(sizeof(int) * NW_WS_SLOTS);
            HZ_CU(cudaMemsetAsync(c->nw_cnt, 0, sizeof(int) * NW_WS_SLOTS, c->st));
        }
        c->kt_begin(cls, pl.bytes, pl.flops);
        launch_gemm_narrow(reinterpret_cast<const GemmProb<float2> *>(pl.d), pl.n, pl.max_tiles32, pl.max_n, split,
                           c->nw_ws, c->nw_cnt, c->st, &c->nl);
        c->kt_end();
        return;
    }
    // FP32 short lists (a sweep step's products) with narrow panels (<= 16 columns):
    // the skinny kernel, whose K loop keeps the next block's loads in flight
    if (sizeof(T2) == 8 && pl.max_n <= 16 && (long long)pl.n * pl.max_tiles32 < GEMM_SPLIT_TILES) {
        c->kt_begin(cls, pl.bytes, pl.flops);
        launch_gemm_skinny<T2>(pl.d, pl.n, pl.max_m, pl.max_n, c->st, &c->nl);
        c->kt_end();
        return;
    }
    // lists of fewer than GEMM_SPLIT_TILES 64 x 32 tiles (a sweep step's products) take
    // 32 x 32 tiles: measured 7-9 % faster on the E+S and 2B-wide W g steps, equal on the
    // others; long lists keep the larger tile
    const bool small = (long long)pl.n * pl.max_tiles < GEMM_SPLIT_TILES;
    const int cfg = small ? 1 : 0, mt = small ? pl.max_tiles32 : pl.max_tiles;
    const int split = gemm_split((long long)pl.n * mt, pl.kmax);
    if (split > 1 && !c->gemm_ws) {
        c->gemm_ws = c->dalloc(sizeof(double2) * 2 * GEMM_SPLIT_TILES * GBM * GBN);
        c->gemm_cnt = (int *)c->dalloc(sizeof(int) * GEMM_SPLIT_TILES);
        HZ_CU(cudaMemsetAsync(c->gemm_cnt, 0, sizeof(int) * GEMM_SPLIT_TILES, c->st));
    }
    c->kt_begin(cls, pl.bytes, pl.flops);
    launch_gemm<T2>(pl.d, pl.n, mt, split, (T2 *)c->gemm_ws, c->gemm_cnt, c->st, &c->nl, cfg);
    c->kt_end();
}

// algorithmic traffic / flops of the chain solves
template <class T2> static void cell_chain_cost(hz_ctx *c, int N, double &bytes, double &flops) {
    const double es = sizeof(T2);
    bytes = flops = 0;
    for (const CellDesc &cd : c->cells) {
        const double nx = cd.nx, nz = cd.nz;
        bytes += es * ((2 * nz - 1) * nx * nx + 2 * (nz - 1) * nx + 4 * nz * nx * N);
        flops += 8.0 * (2 * nz - 1) * nx * nx * N;
    }
}
template <class T2> static void inner_chain_cost(hz_ctx *c, int l0, int nl, int N, double &bytes, double &flops) {
    // the recurrence part (P_j and V_j products); h_j = W_j g_j is counted with the GEMMs
    const double es = sizeof(T2);
    bytes = flops = 0;
    for (int l = l0; l < l0 + nl; l++) {
        const double J = c->C - 1, n2 = 2.0 * c->layers[l].nz;
        if (J <= 1) continue;
        const double ent = 2 * (J - 1) * n2 * n2;
        bytes += es * (ent + 4 * J * n2 * N);
        flops += 8.0 * ent * N;
    }
}

// cell solves of every cell (a1): tensor cores in mixed precision when the
// split blocks were built, else the SIMT chain
template <class T2> static void cell_chain_launch(hz_ctx *c, const CellDesc *d_cells, int ncell, T2 *vol, int N) {
    Ops<T2> &o = ops<T2>(c);
    if constexpr (std::is_same<T2, float2>::value) {
        if (c->wtc) {
            launch_cell_chain_tc(d_cells, ncell, c->wtc, o.cz, vol, N, c->max_nx, c->d_err, c->st, &c->nl);
            return;
        }
    }
    launch_cell_chain<T2>(d_cells, ncell, o.cellW, o.cz, vol, N, c->max_nx, c->st, &c->nl);
}

template <class T2> static void cell_chain(hz_ctx *c, T2 *vol, int N) {
    double by = 0, fl = 0;
    if (c->opts.time_kernels) cell_chain_cost<T2>(c, N, by, fl);
    c->kt_begin(0, by, fl);
    cell_chain_launch<T2>(c, c->d_cells, (int)c->cells.size(), vol, N);
    c->kt_end();
}

// ---------------------------------------------------------- workspace ---
template <class T2> static void build_lists(hz_ctx *c, Work<T2> &W) {
    Ops<T2> &o = ops<T2>(c);
    const int L = c->L, K = L - 1, NX = c->NX, B = W.B;
    const long long rowsz = (long long)NX * B;      // one trace row, B columns
    const long long rowsz2 = (long long)NX * 2 * B; // one trace row, 2B columns
    ListBuilder<T2> lb(c, o);
    auto vec_rows = [&](T2 *base, int k, int comp0) {
        return base + ((long long)k * 4 + comp0) * rowsz;
    };
    // apply M: F from the staged inputs (2B wide), E/S of both sets
    // compressed-block LU: the right-hand sides g_j go to innerH / innerH2, h_j and x_j to inner / inner2
    const bool lr = c->lr_r > 0;
    T2 *gB = lr ? W.innerH : W.inner, *g2B = lr ? W.innerH2 : W.inner2;
    for (int l = 0; l < L; l++) {
        const T2 *in[4];
        for (int q = 0; q < 4; q++) in[q] = W.lin + ((long long)l * 4 + q) * rowsz2;
        lb.add_F(l, 3, in, 2 * B, 2 * B, g2B, 2 * B, 0);
    }
    W.f_full = lb.finish();
    for (int l = 0; l < L; l++) {
        const T2 *in[4];
        T2 *out[4];
        for (int q = 0; q < 4; q++) {
            in[q] = W.lin + ((long long)l * 4 + q) * rowsz2;
            out[q] = W.lout + ((long long)l * 4 + q) * rowsz2;
        }
        if (l < L - 1) lb.add_ES(l, 3, in, 2 * B, 2, out, 2 * B, W.inner2, 2 * B, B, 0);  // set A -> rows n, n+1
        if (l > 0) {
            const T2 *inB[4];
            T2 *outB[4];
            for (int q = 0; q < 4; q++) {
                inB[q] = in[q] + B;
                outB[q] = out[q] + B;
            }
            // set B -> rows 0, 1 (E reads the inner traces of columns B..2B)
            lb.add_ES(l, 3, inB, 2 * B, 1, outB, 2 * B, W.inner2 + B, 2 * B, B, 0);
        }
    }
    W.es_bot_A = lb.finish();
    // downward sweep on pb: layer k from the d-part of interface k-1 into the d-part of interface k
    W.f_down.assign(L, ProbList<T2>());
    W.es_down.assign(L, ProbList<T2>());
    for (int k = 1; k <= L - 2; k++) {
        const T2 *in[4] = {vec_rows(W.pb, k - 1, 0), vec_rows(W.pb, k - 1, 1), nullptr, nullptr};
        lb.add_F(k, 1, in, B, B, gB, B, 0);
        W.f_down[k] = lb.finish();
        T2 *out[4] = {nullptr, nullptr, vec_rows(W.pb, k, 0), vec_rows(W.pb, k, 1)};
        lb.add_ES(k, 1, in, B, 2, out, B, W.inner, B, B, 1);
        W.es_down[k] = lb.finish();
    }
    // the same downward steps through the composites (compressed-block LU)
    const bool comp = lr && o.CP2 && o.LAM;
    if (comp) {  // the polarized operator: set A (columns 0..B) -> rows n, n+1, set B -> rows 0, 1
        for (int l = 0; l < L; l++) {
            const T2 *in[4], *inB[4];
            T2 *out[4], *outB[4];
            for (int q = 0; q < 4; q++) {
                in[q] = W.lin + ((long long)l * 4 + q) * rowsz2;
                out[q] = W.lout + ((long long)l * 4 + q) * rowsz2;
                inB[q] = in[q] + B;
                outB[q] = out[q] + B;
            }
            if (l < L - 1) lb.add_compP2(l, 0, 4, in, 2 * B, 2, out, 2 * B, B, 0);
            if (l > 0) lb.add_compP2(l, 0, 4, inB, 2 * B, 0, outB, 2 * B, B, 0);
            lb.add_compP1(l, 0, 4, in, 2 * B, W.ac2, 2 * B, B);
            lb.add_compP1(l, 0, 4, inB, 2 * B, W.ac2 + B, 2 * B, B);
        }
        W.cA_M = lb.finish();
        for (int l = 0; l < L; l++) {
            T2 *out[4], *outB[4];
            for (int q = 0; q < 4; q++) {
                out[q] = W.lout + ((long long)l * 4 + q) * rowsz2;
                outB[q] = out[q] + B;
            }
            if (l < L - 1) lb.add_compC(l, 2, out, 2 * B, W.ts2, 2 * B, B);
            if (l > 0) lb.add_compC(l, 0, outB, 2 * B, W.ts2 + B, 2 * B, B);
        }
        W.cC_M = lb.finish();
        W.cA_down.assign(L, ProbList<T2>());
        W.cC_down.assign(L, ProbList<T2>());
        for (int k = 1; k <= L - 2; k++) {
            const T2 *in[4] = {vec_rows(W.pb, k - 1, 0), vec_rows(W.pb, k - 1, 1), nullptr, nullptr};
            T2 *out[4] = {nullptr, nullptr, vec_rows(W.pb, k, 0), vec_rows(W.pb, k, 1)};
            lb.add_compA(k, 0, 2, in, B, 2, out, B, W.ac, B);
            W.cA_down[k] = lb.finish();
            lb.add_compC(k, 2, out, B, W.ts, B, B);
            W.cC_down[k] = lb.finish();
        }
    }
    // upward sweep on pb: layer k+1 from the u-part of interface k+1 into the u-part of interface k
    W.f_up.assign(L, ProbList<T2>());
    W.es_up.assign(L, ProbList<T2>());
    for (int k = L - 3; k >= 0; k--) {
        const T2 *in[4] = {nullptr, nullptr, vec_rows(W.pb, k + 1, 2), vec_rows(W.pb, k + 1, 3)};
        lb.add_F(k + 1, 2, in, B, B, gB, B, 0);
        W.f_up[k] = lb.finish();
        T2 *out[4] = {vec_rows(W.pb, k, 2), vec_rows(W.pb, k, 3), nullptr, nullptr};
        lb.add_ES(k + 1, 2, in, B, 1, out, B, W.inner, B, B, 1);
        W.es_up[k] = lb.finish();
    }
    if (comp) {
        W.cA_up.assign(L, ProbList<T2>());
        W.cC_up.assign(L, ProbList<T2>());
        for (int k = L - 3; k >= 0; k--) {
            const T2 *in[4] = {nullptr, nullptr, vec_rows(W.pb, k + 1, 2), vec_rows(W.pb, k + 1, 3)};
            T2 *out[4] = {vec_rows(W.pb, k, 2), vec_rows(W.pb, k, 3), nullptr, nullptr};
            lb.add_compA(k + 1, 2, 2, in, B, 0, out, B, W.ac, B);
            W.cA_up[k] = lb.finish();
            lb.add_compC(k + 1, 0, out, B, W.ts, B, B);
            W.cC_up[k] = lb.finish();
        }
    }
    // reflections on pb: layer k+1, top = d of interface k, bottom = d of interface k+1
    for (int k = 0; k < K; k++) {
        int mask = (k + 1 <= L - 2) ? 3 : 1;
        const T2 *in[4] = {vec_rows(W.pb, k, 0), vec_rows(W.pb, k, 1), nullptr, nullptr};
        if (mask & 2) {
            in[2] = vec_rows(W.pb, k + 1, 0);
            in[3] = vec_rows(W.pb, k + 1, 1);
        }
        lb.add_F(k + 1, mask, in, B, B, gB, B, 0);
    }
    W.f_refl = lb.finish();
    for (int k = 0; k < K; k++) {
        int mask = (k + 1 <= L - 2) ? 3 : 1;
        const T2 *in[4] = {vec_rows(W.pb, k, 0), vec_rows(W.pb, k, 1), nullptr, nullptr};
        if (mask & 2) {
            in[2] = vec_rows(W.pb, k + 1, 0);
            in[3] = vec_rows(W.pb, k + 1, 1);
        }
        T2 *out[4] = {vec_rows(W.pb, k, 2), vec_rows(W.pb, k, 3), nullptr, nullptr};
        lb.add_ES(k + 1, mask, in, B, 1, out, B, W.inner, B, B, 1);
    }
    W.es_refl = lb.finish();
    if (comp) {  // the same reflections through the composites: [P2, P1] lists, then P3
        for (int k = 0; k < K; k++) {
            const int nq = (k + 1 <= L - 2) ? 4 : 2;
            const T2 *in[4] = {vec_rows(W.pb, k, 0), vec_rows(W.pb, k, 1), nullptr, nullptr};
            if (nq == 4) {
                in[2] = vec_rows(W.pb, k + 1, 0);
                in[3] = vec_rows(W.pb, k + 1, 1);
            }
            T2 *out[4] = {vec_rows(W.pb, k, 2), vec_rows(W.pb, k, 3), nullptr, nullptr};
            lb.add_compA(k + 1, 0, nq, in, B, 0, out, B, W.ac, B);
        }
        W.cA_refl = lb.finish();
        for (int k = 0; k < K; k++) {
            T2 *out[4] = {vec_rows(W.pb, k, 2), vec_rows(W.pb, k, 3), nullptr, nullptr};
            lb.add_compC(k + 1, 0, out, B, W.ts, B, B);
        }
        W.cC_refl = lb.finish();
    }
    // reconstruction F-step from the traces tr = pc viewed as [K][2][NX][B] (accumulating)
    for (int l = 0; l < L; l++) {
        int mask = (l > 0 ? 1 : 0) | (l < L - 1 ? 2 : 0);
        const T2 *in[4] = {nullptr, nullptr, nullptr, nullptr};
        if (l > 0) {
            in[0] = W.pc + ((long long)(l - 1) * 2 + 0) * rowsz;
            in[1] = W.pc + ((long long)(l - 1) * 2 + 1) * rowsz;
        }
        if (l < L - 1) {
            in[2] = W.pc + ((long long)l * 2 + 0) * rowsz;
            in[3] = W.pc + ((long long)l * 2 + 1) * rowsz;
        }
        if (mask) lb.add_F(l, mask, in, B, B, gB, B, 1);
    }
    W.f_rec = lb.finish();
    // Newton samples: lout (B-wide view [L][4][NX][B]) += E x_f
    for (int l = 0; l < L; l++) {
        T2 *out[4];
        for (int q = 0; q < 4; q++) out[q] = W.lout + ((long long)l * 4 + q) * rowsz;
        const T2 *in[4] = {nullptr, nullptr, nullptr, nullptr};
        lb.add_ES(l, 0, in, B, 3, out, B, W.inner, B, B, 1);
    }
    W.e_newton = lb.finish();
    // h_j = W_j g_j for every interface, ordered by layer (B wide and 2B wide)
    W.hoff.assign(L + 1, 0);
    W.hbytes.assign(L, 0.0);
    W.hflops.assign(L, 0.0);
    W.htiles.assign(L, 0);
    W.utiles.assign(L, 0);
    for (int wide = 0; wide < 2; wide++) {
        const int Bw = wide ? 2 * B : B;
        // dense: h_j = W_j g_j from inner into innerH; compressed: from innerH into inner,
        // with ac_j = STW_j g_j beside it
        T2 *gin = lr ? (wide ? W.innerH2 : W.innerH) : (wide ? W.inner2 : W.inner);
        T2 *hout = lr ? (wide ? W.inner2 : W.inner) : (wide ? W.innerH2 : W.innerH);
        T2 *acv = wide ? W.ac2 : W.ac;
        const int r = c->lr_r;
        int cnt = 0;
        for (int l = 0; l < L; l++) {
            const LayerDesc &ld = c->layers[l];
            const int n2 = 2 * ld.nz;
            if (!wide) W.hoff[l] = cnt;
            double b0 = lb.bytes, f0 = lb.flops;
            const long long t0 = lb.tiles32;
            for (int j = 0; j < c->C - 1; j++) {
                GemmProb<T2> g{};
                g.A = o.W + ld.W_off + (long long)j * n2 * n2;
                g.lda = n2;
                g.M = n2;
                g.K = n2;
                g.N = Bw;
                g.xseg = g.yseg = 1 << 30;
                g.ldx = g.ldy = Bw;
                g.X[0] = gin + (ld.inner_off + (long long)(j + 1) * n2) * Bw;
                g.Y[0] = hout + (ld.inner_off + (long long)(j + 1) * n2) * Bw;
                g.beta = 0;
                g.alpha = 1.f;
                lb.push(g);
                cnt++;
                if (lr) {
                    g.A = o.STW + ld.lr_off + (long long)j * 2 * r * n2;
                    g.M = 2 * r;
                    g.Y[0] = acv + (ld.ac_off + (long long)j * 2 * r) * Bw;
                    lb.push(g);
                    cnt++;
                }
            }
            if (!wide) {
                W.hbytes[l] = lb.bytes - b0;
                W.hflops[l] = lb.flops - f0;
                W.htiles[l] = lb.tiles32 - t0;
            }
        }
        if (!wide) W.hoff[L] = cnt;
        if (wide)
            W.h2B = lb.finish();
        else
            W.hB = lb.finish();
    }
    // compressed-block LU: x_j += UX_j ts_j, ordered by layer
    if (lr) {
        W.uoff.assign(L + 1, 0);
        const int r = c->lr_r;
        for (int wide = 0; wide < 2; wide++) {
            const int Bw = wide ? 2 * B : B;
            T2 *xv = wide ? W.inner2 : W.inner;
            T2 *tsv = wide ? W.ts2 : W.ts;
            int cnt = 0;
            for (int l = 0; l < L; l++) {
                const LayerDesc &ld = c->layers[l];
                const int n2 = 2 * ld.nz;
                if (!wide) W.uoff[l] = cnt;
                const long long t0 = lb.tiles32;
                for (int j = 0; j < c->C - 1; j++) {
                    GemmProb<T2> g{};
                    g.A = o.UX + ld.lr_off + (long long)j * n2 * 2 * r;
                    g.lda = 2 * r;
                    g.M = n2;
                    g.K = 2 * r;
                    g.N = Bw;
                    g.xseg = g.yseg = 1 << 30;
                    g.ldx = g.ldy = Bw;
                    g.X[0] = tsv + (ld.ac_off + (long long)j * 2 * r) * Bw;
                    g.Y[0] = xv + (ld.inner_off + (long long)(j + 1) * n2) * Bw;
                    g.beta = 1;
                    g.alpha = 1.f;
                    lb.push(g);
                    cnt++;
                }
                if (!wide) W.utiles[l] = lb.tiles32 - t0;
            }
            if (!wide) W.uoff[L] = cnt;
            if (wide)
                W.ux2B = lb.finish();
            else
                W.uxB = lb.finish();
        }
        // ts = LAM ac, one problem per layer
        const int Nc = 2 * r * (c->C - 1);
        for (int wide = 0; wide < 2; wide++) {
            const int Bw = wide ? 2 * B : B;
            for (int l = 0; l < L; l++) {
                const LayerDesc &ld = c->layers[l];
                GemmProb<T2> g{};
                g.A = o.LAM + ld.lam_off;
                g.lda = Nc;
                g.M = Nc;
                g.K = Nc;
                g.N = Bw;
                g.xseg = g.yseg = 1 << 30;
                g.ldx = g.ldy = Bw;
                g.X[0] = (wide ? W.ac2 : W.ac) + ld.ac_off * Bw;
                g.Y[0] = (wide ? W.ts2 : W.ts) + ld.ac_off * Bw;
                g.beta = 0;
                g.alpha = 1.f;
                lb.push(g);
            }
            if (wide)
                W.lam2B = lb.finish();
            else
                W.lamB = lb.finish();
        }
    }
    // single-layer applications (component entry point), inputs/outputs in lin/lout (B wide)
    W.f_layer.assign(L, ProbList<T2>());
    W.es_layer.assign(L, ProbList<T2>());
    for (int l = 0; l < L; l++) {
        const T2 *in[4];
        T2 *out[4];
        for (int q = 0; q < 4; q++) {
            in[q] = W.lin + ((long long)l * 4 + q) * rowsz;
            out[q] = W.lout + ((long long)l * 4 + q) * rowsz;
        }
        lb.add_F(l, 3, in, B, B, gB, B, 0);
        W.f_layer[l] = lb.finish();
        lb.add_ES(l, 3, in, B, 3, out, B, W.inner, B, B, 0);
        W.es_layer[l] = lb.finish();
    }
}

// K slices of a narrow list for a launch of `wave` co-resident CTAs (the rule of run())
static int narrow_split(long long n, int max_tiles32, long long tiles32, int kmax, long long wave) {
    const long long slots = n * max_tiles32;
    const int nbk = (kmax + NW_KB - 1) / NW_KB;
    if (tiles32 <= 0 || slots > NW_WS_SLOTS) return 1;
    return (int)std::max(1LL, std::min<long long>({8, wave / tiles32, NW_WS_SLOTS / slots,
                                                   std::max(1, nbk / (2 * NW_WPC))}));
}

// phases of the persistent downward / upward sweeps (compressed-block LU composites,
// FP32, batches of <= 16 even columns): per step [P2, P1], Λ, P3
template <class T2> static void build_sweep_phases(hz_ctx *c, Work<T2> &W) {
    if constexpr (!std::is_same<T2, float2>::value) {
        return;
    } else {
        // opt-in (HZ_PERSIST=1, read when a workspace is built): on the 2000 x 4000 workload the
        // persistent sweeps measured 270.4 ms per step against 267.0 with one launch per list
        const char *pe = getenv("HZ_PERSIST");
        const bool on = pe && strcmp(pe, "1") == 0;
        const int L = c->L, B = W.B;
        if (!on || W.cA_down.empty() || B > NW_NB || (B & 1) || L < 3) return;
        const int grid = narrow_sweep_grid();
        if (grid <= 0) return;
        bool split_ws = false;
        auto phase = [&](const ProbList<float2> &pl, std::vector<NwPhase> &v, double &by, double &fl) {
            if (!pl.n) return true;
            if (pl.max_n > NW_NB) return false;
            NwPhase q{pl.d, pl.n, pl.max_tiles32, narrow_split(pl.n, pl.max_tiles32, pl.tiles32, pl.kmax, grid)};
            split_ws |= q.split > 1;
            v.push_back(q);
            by += pl.bytes;
            fl += pl.flops;
            return true;
        };
        auto lam = [&](int l) {
            ProbList<float2> ls = W.lamB;
            ls.d = W.lamB.d + l;
            ls.n = 1;
            ls.tiles32 = W.lamB.max_tiles32;
            ls.bytes = W.lamB.bytes / L;
            ls.flops = W.lamB.flops / L;
            return ls;
        };
        std::vector<NwPhase> dn, up;
        bool ok = true;
        for (int k = 1; k <= L - 2 && ok; k++)
            ok = phase(W.cA_down[k], dn, W.sw_bytes[0], W.sw_flops[0]) &&
                 phase(lam(k), dn, W.sw_bytes[0], W.sw_flops[0]) &&
                 phase(W.cC_down[k], dn, W.sw_bytes[0], W.sw_flops[0]);
        for (int k = L - 3; k >= 0 && ok; k--)
            ok = phase(W.cA_up[k], up, W.sw_bytes[1], W.sw_flops[1]) &&
                 phase(lam(k + 1), up, W.sw_bytes[1], W.sw_flops[1]) &&
                 phase(W.cC_up[k], up, W.sw_bytes[1], W.sw_flops[1]);
        if (!ok || dn.empty() || up.empty()) return;
        if (split_ws && !c->nw_ws) {
            c->nw_ws = (float2 *)c->dalloc(sizeof(float2) * (size_t)NW_WS_SLOTS * 32 * NW_NB);
            c->nw_cnt = (int *)c->dalloc(sizeof(int) * NW_WS_SLOTS);
            HZ_CU(cudaMemsetAsync(c->nw_cnt, 0, sizeof(int) * NW_WS_SLOTS, c->st));
        }
        W.sw_down = (NwPhase *)c->dalloc(sizeof(NwPhase) * dn.size());
        W.sw_up = (NwPhase *)c->dalloc(sizeof(NwPhase) * up.size());
        W.sw_bar = (unsigned *)c->dalloc(sizeof(unsigned));
        HZ_CU(cudaMemcpy(W.sw_down, dn.data(), sizeof(NwPhase) * dn.size(), cudaMemcpyHostToDevice));
        HZ_CU(cudaMemcpy(W.sw_up, up.data(), sizeof(NwPhase) * up.size(), cudaMemcpyHostToDevice));
        W.nsw_down = (int)dn.size();
        W.nsw_up = (int)up.size();
    }
}

template <class T2> static std::unique_ptr<Work<T2>> &work_slot(hz_ctx *c);
template <> std::unique_ptr<Work<double2>> &work_slot<double2>(hz_ctx *c) { return c->w64; }
template <> std::unique_ptr<Work<float2>> &work_slot<float2>(hz_ctx *c) { return c->w32; }

template <class T2> static void free_work(hz_ctx *c, Work<T2> &W) {
    void *ptrs[] = {W.vol, W.vol2, W.inner, W.inner2, W.inner_f, W.innerH, W.innerH2, W.ac, W.ts, W.ac2, W.ts2, W.lin, W.lout, W.pa, W.pb, W.pc, W.Z, W.V, W.w64,
                    W.rhs64, W.x64, W.dots, W.hbuf, W.gsrc, W.u, W.io, W.rnorm};
    for (void *q : ptrs) c->dfree(q);
    auto fl = [&](ProbList<T2> &pl) { c->dfree(pl.d); };
    fl(W.f_full);
    fl(W.es_bot_A);
    fl(W.f_refl);
    fl(W.es_refl);
    fl(W.f_rec);
    fl(W.e_newton);
    fl(W.hB);
    fl(W.h2B);
    fl(W.uxB);
    fl(W.ux2B);
    fl(W.lamB);
    fl(W.cA_refl);
    fl(W.cA_M);
    c->dfree(W.sw_down);
    c->dfree(W.sw_up);
    c->dfree(W.sw_bar);
    fl(W.cC_M);
    fl(W.cC_refl);
    fl(W.lam2B);
    for (auto *vv : {&W.f_down, &W.es_down, &W.f_up, &W.es_up, &W.f_layer, &W.es_layer, &W.cA_down, &W.cC_down,
                     &W.cA_up, &W.cC_up})
        for (auto &pl : *vv) fl(pl);
    if (W.hhost) cudaFreeHost(W.hhost);
    if (W.rhost) cudaFreeHost(W.rhost);
}

template <class T2> Work<T2> &work(hz_ctx *c, int B) {
    auto &slot = work_slot<T2>(c);
    // FGMRES keeps restart+1 basis vectors; Bi-CGstab uses 6 of them and 14 B host slots
    const int m = std::max(c->opts.krylov == HZ_BICGSTAB ? 6 : 1, c->opts.restart);
    if (slot && slot->B == B && slot->restart == m) return *slot;
    if (slot) {
        free_work(c, *slot);
        slot.reset();
    }
    slot.reset(new Work<T2>());
    Work<T2> &W = *slot;
    W.B = B;
    W.restart = m;
    const long long ntr = c->n_tr(), N = (long long)c->NX * c->NZ;
    auto al = [&](long long n, size_t es) { return c->dalloc(es * std::max(n, 1LL)); };
    W.vol = (T2 *)al(c->tot_vol * B, sizeof(T2));
    W.vol2 = (T2 *)al(c->tot_vol * B, sizeof(T2));
    W.inner = (T2 *)al(c->tot_inner * B, sizeof(T2));
    W.inner2 = (T2 *)al(c->tot_inner * 2 * B, sizeof(T2));
    W.inner_f = (T2 *)al(c->tot_inner * B, sizeof(T2));
    W.innerH = (T2 *)al(c->tot_inner * B, sizeof(T2));
    W.innerH2 = (T2 *)al(c->tot_inner * 2 * B, sizeof(T2));
    if (c->lr_r > 0) {
        W.ac = (T2 *)al(c->tot_ac * B, sizeof(T2));
        W.ts = (T2 *)al(c->tot_ac * B, sizeof(T2));
        W.ac2 = (T2 *)al(c->tot_ac * 2 * B, sizeof(T2));
        W.ts2 = (T2 *)al(c->tot_ac * 2 * B, sizeof(T2));
        HZ_CU(cudaMemsetAsync(W.ts, 0, sizeof(T2) * c->tot_ac * B, c->st));
        HZ_CU(cudaMemsetAsync(W.ts2, 0, sizeof(T2) * c->tot_ac * 2 * B, c->st));
    }
    HZ_CU(cudaMemsetAsync(W.inner, 0, sizeof(T2) * c->tot_inner * B, c->st));
    HZ_CU(cudaMemsetAsync(W.inner2, 0, sizeof(T2) * c->tot_inner * 2 * B, c->st));
    HZ_CU(cudaMemsetAsync(W.inner_f, 0, sizeof(T2) * c->tot_inner * B, c->st));
    W.lin = (T2 *)al((long long)c->L * 4 * c->NX * 2 * B, sizeof(T2));
    W.lout = (T2 *)al((long long)c->L * 4 * c->NX * 2 * B, sizeof(T2));
    HZ_CU(cudaMemsetAsync(W.lout, 0, sizeof(T2) * c->L * 4 * c->NX * 2 * B, c->st));
    W.pa = (T2 *)al(ntr * B, sizeof(T2));
    W.pb = (T2 *)al(ntr * B, sizeof(T2));
    W.pc = (T2 *)al(ntr * B, sizeof(T2));
    W.Z = (T2 *)al((long long)m * ntr * B, sizeof(T2));
    W.V = (double2 *)al((long long)(m + 1) * ntr * B, sizeof(double2));
    W.w64 = (double2 *)al(ntr * B, sizeof(double2));
    W.rhs64 = (double2 *)al(ntr * B, sizeof(double2));
    W.x64 = (double2 *)al(ntr * B, sizeof(double2));
    W.dots = (double *)al((long long)(m + 2) * dots_chunks(c->n_tr(), B) * B * 2, sizeof(double));
    W.hbuf = (double *)al((long long)(2 * m + 4) * B * 2, sizeof(double));
    HZ_CU(cudaMallocHost(&W.hhost, sizeof(double) * (2 * m + 4) * B * 2));
    W.gsrc = (double2 *)al(N * B, sizeof(double2));
    W.u = (double2 *)al(N * B, sizeof(double2));
    W.io = (double2 *)al(N * B, sizeof(double2));
    W.rnorm = (double *)al((long long)4096 * B + 4 * B, sizeof(double));
    HZ_CU(cudaMallocHost(&W.rhost, sizeof(double) * 4 * B));
    build_lists(c, W);
    build_sweep_phases(c, W);
    return W;
}
template Work<double2> &work<double2>(hz_ctx *, int);
template Work<float2> &work<float2>(hz_ctx *, int);

// ------------------------------------------------------- layer pieces ---
// inner solve of layers [l0, l0+nl): h_j = W_j g_j (batched GEMM) then the
// block-LU recurrences; `wide` selects the 2B-wide buffers of the polarized operator
// ts = LAM ac for layers [l0, l0 + nl) (compressed-block LU), one product per layer
template <class T2> static void run_lam(hz_ctx *c, Work<T2> &W, bool wide, int l0, int nl) {
    const ProbList<T2> &la = wide ? W.lam2B : W.lamB;
    ProbList<T2> ls = la;
    ls.d = la.d + l0;
    ls.n = nl;
    ls.tc_tiles = (long long)nl * la.tc_max_tiles;
    ls.tiles32 = (long long)nl * la.max_tiles32;
    ls.bytes = la.bytes * nl / c->L;
    ls.flops = la.flops * nl / c->L;
    run(c, ls, 1);
}

// the compressed-block LU recursion ts = LAM ac of layers [l0, l0 + nl): one product for a
// single layer, else the r-vector chain kernel over the layers
template <class T2> static void lr_recursion(hz_ctx *c, Work<T2> &W, bool wide, int l0, int nl) {
    const int N = wide ? 2 * W.B : W.B;
    if (nl == 1 || !lr_chain_fits<T2>(c, N)) {
        run_lam(c, W, wide, l0, nl);
        return;
    }
    double by = 0, fl = 0;
    if (c->opts.time_kernels) {
        const double J = c->C - 1, es = sizeof(T2), r = c->lr_r;
        by = nl * es * (3 * J * r * r + 4 * J * r * N);
        fl = nl * 8.0 * 3 * J * r * r * N;
    }
    c->kt_begin(1, by, fl);
    launch_lr_chain<T2>(c, c->d_layer_ids + l0, nl, ops<T2>(c).MRN, wide ? W.ac2 : W.ac, wide ? W.ts2 : W.ts, N);
    c->kt_end();
}

template <class T2> static void chain_layers(hz_ctx *c, Work<T2> &W, bool wide, int l0, int nl) {
    if (c->C < 2) return;
    Ops<T2> &o = ops<T2>(c);
    const ProbList<T2> &all = wide ? W.h2B : W.hB;
    ProbList<T2> sub = all;
    sub.d = all.d + W.hoff[l0];
    sub.n = W.hoff[l0 + nl] - W.hoff[l0];
    sub.tc_tiles = (long long)sub.n * all.tc_max_tiles;
    sub.bytes = sub.flops = 0;
    sub.tiles32 = 0;
    for (int l = l0; l < l0 + nl; l++) {
        sub.bytes += W.hbytes[l] * (wide ? 2 : 1);
        sub.flops += W.hflops[l] * (wide ? 2 : 1);
        sub.tiles32 += W.htiles[l];
    }
    run(c, sub);
    const int N = wide ? 2 * W.B : W.B;
    double by = 0, fl = 0;
    if (c->lr_r > 0) {  // compressed-block LU: the r-vector recursion, then x_j += UX_j ts_j
        const int r = c->lr_r;
        if (c->opts.time_kernels)
            for (int l = l0; l < l0 + nl; l++) {
                const double J = c->C - 1, es = sizeof(T2);
                by += es * (3 * J * r * r + 4 * J * r * N);
                fl += 8.0 * 3 * J * r * r * N;
            }
        if (nl == 1 || !lr_chain_fits<T2>(c, N)) {
            // one layer (a sweep step): the recursion as one product, ts = LAM ac, instead
            // of 2(C-1) dependent steps on a few SMs
            run_lam(c, W, wide, l0, nl);
        } else {
            c->kt_begin(1, by, fl);
            launch_lr_chain<T2>(c, c->d_layer_ids + l0, nl, o.MRN, wide ? W.ac2 : W.ac, wide ? W.ts2 : W.ts, N);
            c->kt_end();
        }
        const ProbList<T2> &ua = wide ? W.ux2B : W.uxB;
        ProbList<T2> us = ua;
        us.d = ua.d + W.uoff[l0];
        us.n = W.uoff[l0 + nl] - W.uoff[l0];
        us.tc_tiles = (long long)us.n * ua.tc_max_tiles;
        us.bytes = us.flops = 0;
        us.tiles32 = 0;
        for (int l = l0; l < l0 + nl; l++) {
            us.tiles32 += W.utiles[l];
            const double n2 = 2.0 * c->layers[l].nz, J = c->C - 1, es = sizeof(T2);
            us.bytes += es * J * (n2 * 2 * r + 2 * r * N + 2 * n2 * N);
            us.flops += 8.0 * J * n2 * 2 * r * N;
        }
        run(c, us);
        return;
    }
    if (c->opts.time_kernels) inner_chain_cost<T2>(c, l0, nl, N, by, fl);
    c->kt_begin(1, by, fl);
    launch_inner_sweep<T2>(c->d_layers, c->d_layer_ids + l0, nl, o.P, o.V, wide ? W.innerH2 : W.innerH,
                           wide ? W.inner2 : W.inner, N, 2 * c->max_nz, c->d_err, c->st, &c->nl,
                           c->opts.autotune != 0);
    c->kt_end();
}

template <class T2> static void nested_apply_M(hz_ctx *c, Work<T2> &W, const T2 *x, double2 *y);
template <class T2> static void nested_precond(hz_ctx *c, Work<T2> &W, int kind);

// polarized operator: y (FP64) = M x (x in the working precision)
// HZ_SWEEP=factored keeps the sweep steps and the polarized operator on the factored operators (for comparisons)
static bool comp_off() {
    static const bool off = getenv("HZ_SWEEP") && strcmp(getenv("HZ_SWEEP"), "factored") == 0;
    return off;
}

template <class T2> static void apply_M(hz_ctx *c, Work<T2> &W, const T2 *x, double2 *y) {
    if (c->nested()) return nested_apply_M(c, W, x, y);
    const int B = W.B;
    const long long n = (long long)c->L * 4 * c->NX * 2 * B;
    k_stage_M<T2><<<grid1(n), 256, 0, c->st>>>(x, W.lin, c->L, c->NX, B);
    HZ_CU(cudaGetLastError());
    c->nl++;
    if (!W.cA_M.d || comp_off()) {
        run(c, W.f_full);
        chain_layers(c, W, true, 0, c->L);
        run(c, W.es_bot_A);
    } else {  // through the composites (compressed-block LU)
        run(c, W.cA_M);
        lr_recursion(c, W, true, 0, c->L);
        run(c, W.cC_M);
    }
    const long long m = c->n_tr() * B;
    k_combine_M<T2><<<grid1(m), 256, 0, c->st>>>(x, W.lout, y, c->L, c->NX, B);
    HZ_CU(cudaGetLastError());
    c->nl++;
}

// preconditioner on W.pb in place (input copied there by the caller):
// kind 0 GS, 1 Jacobi, 2 down only, 3 up only, 4 reflections only

template <class T2> static void precond_inplace(hz_ctx *c, Work<T2> &W, int kind) {
    if (c->nested()) return nested_precond(c, W, kind);
    const int L = c->L;
    // a sweep step through the composites (compressed-block LU): three products
    const bool comp = !W.cA_down.empty() && !comp_off();
    // the whole sweep as one persistent launch (a context solving alone on the GPU)
    const bool persist = comp && W.nsw_down > 0 && c->group_n <= 1 && !c->parent && c->lanes.empty();
    auto sweep = [&](int dir) {
        c->kt_begin(2, W.sw_bytes[dir], W.sw_flops[dir]);
        launch_narrow_sweep(dir ? W.sw_up : W.sw_down, dir ? W.nsw_up : W.nsw_down, c->nw_ws, c->nw_cnt, W.sw_bar,
                            c->d_err, narrow_sweep_grid(), c->st, &c->nl);
        c->kt_end();
    };
    if ((kind == 0 || kind == 1 || kind == 2) && persist) {
        sweep(0);
    } else if (kind == 0 || kind == 1 || kind == 2) {
        for (int k = 1; k <= L - 2; k++) {
            if (comp) {
                run(c, W.cA_down[k]);
                run_lam(c, W, false, k, 1);
                run(c, W.cC_down[k]);
                continue;
            }
            run(c, W.f_down[k]);
            chain_layers(c, W, false, k, 1);
            run(c, W.es_down[k]);
        }
    }
    if (kind == 0 || kind == 4) {
        if (kind == 4) {  // u := 0 so that the step below leaves -L d in the u-part
            const long long rowsz = (long long)c->NX * W.B;
            for (int k = 0; k < L - 1; k++)
                HZ_CU(cudaMemsetAsync(W.pb + ((long long)k * 4 + 2) * rowsz, 0, sizeof(T2) * 2 * rowsz, c->st));
        }
        // w = v_u - L d = v_u + [t0, t1 - d_b]: subtract d_b here, add t below
        k_gs_fix<T2><<<grid1((long long)(L - 1) * c->NX * W.B), 256, 0, c->st>>>(W.pb, L - 1, c->NX, W.B);
        HZ_CU(cudaGetLastError());
        c->nl++;
        if (comp) {
            run(c, W.cA_refl);
            lr_recursion(c, W, false, 1, L - 1);
            run(c, W.cC_refl);
        } else {
            run(c, W.f_refl);
            chain_layers(c, W, false, 1, L - 1);
            run(c, W.es_refl);
        }
        if (kind == 4) {
            k_refl_finish<T2><<<grid1((long long)(L - 1) * c->NX * W.B), 256, 0, c->st>>>(W.pb, L - 1, c->NX, W.B);
            HZ_CU(cudaGetLastError());
            c->nl++;
        }
    }
    if ((kind == 0 || kind == 1 || kind == 3) && persist) {
        sweep(1);
    } else if (kind == 0 || kind == 1 || kind == 3) {
        for (int k = L - 3; k >= 0; k--) {
            if (comp) {
                run(c, W.cA_up[k]);
                run_lam(c, W, false, k + 1, 1);
                run(c, W.cC_up[k]);
                continue;
            }
            run(c, W.f_up[k]);
            chain_layers(c, W, false, k + 1, 1);
            run(c, W.es_up[k]);
        }
    }
}


// ------------------------------------------ inner nested polarized traces ---
// (opts.inner = HZ_INNER_NESTED, Section 4.2.)  A layer's local problem with x
// and z swapped is a problem of the same form whose layers are the cells, so
// the layer's inner context (hz_factor builds one per layer, with a lane for
// 2B-wide applications) solves it with its own FGMRES on the cells' polarized
// traces, preconditioned by the Gauss-Seidel sweeps over the cells.  Every
// local solve of the online stage goes through these inner solves: the source
// volume of each listed layer (its part of the source and the Appendix C
// forcing of trace rows 0, 1, n, n+1, symmetric form) on the transposed layer
// grid [Bw][NX][nz_l] -> the inner solves of the listed layers as one lockstep
// group -> samples at rows 0, 1, n, n+1 and / or the owned rows added to the
// global field.

// f[b][x][r] of layer ld: vsrc ([N][B], rows ld.s + r, owned rows only) and the
// forcing of in ([4][NX][Bw]: rows 0, 1, n, n+1; null: none)
template <class T2>
__global__ void k_nested_src(LayerDesc ld, const T2 *__restrict__ in, const double2 *__restrict__ vsrc,
                             const double2 *__restrict__ ggam, int NX, int Bw, int B, int p, double2 *f) {
    const int nz = ld.nz;
    const long long rowsz = (long long)NX * Bw, n = (long long)Bw * NX * nz;
    const int r0 = p - 1, r1 = p, rn = p + ld.n - 1, rn1 = p + ld.n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e % nz);
        const long long q = e / nz;
        const int x = (int)(q % NX), b = (int)(q / NX);
        double2 v = make_double2(0.0, 0.0);
        if (vsrc && r >= ld.row_lo && r < ld.row_hi) v = vsrc[((long long)(ld.s + r) * NX + x) * B + b];
        if (in && (r == r0 || r == r1 || r == rn || r == rn1)) {
            const long long ix = (long long)x * Bw + b;
            double2 s = make_double2(0.0, 0.0);
            if (r == r0) s = s + to2(in[rowsz + ix], double2{});       // row 0  <- +gamma t(row 1)
            if (r == r1) s = s - to2(in[ix], double2{});               // row 1  <- -gamma t(row 0)
            if (r == rn) s = s - to2(in[3 * rowsz + ix], double2{});   // row n  <- -gamma t(row n+1)
            if (r == rn1) s = s + to2(in[2 * rowsz + ix], double2{});  // row n+1 <- +gamma t(row n)
            v = v + ggam[x] * s;
        }
        f[e] = v;
    }
}

// samples of u[b][x][r] at rows 0, 1, n, n+1 into out ([4][NX][Bw]), and the
// owned rows added to uacc ([N][B], Bw == B)
template <class T2>
__global__ void k_nested_out(LayerDesc ld, const double2 *__restrict__ u, T2 *out, double2 *uacc, int NX, int Bw,
                             int B, int p) {
    const int nz = ld.nz;
    const long long rowsz = (long long)NX * Bw;
    const long long stride = (long long)gridDim.x * blockDim.x, e0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (out) {
        for (long long e = e0; e < 4 * rowsz; e += stride) {
            const int q = (int)(e / rowsz);
            const long long rem = e % rowsz;
            const int x = (int)(rem / Bw), b = (int)(rem % Bw);
            const int r = q == 0 ? p - 1 : (q == 1 ? p : (q == 2 ? p + ld.n - 1 : p + ld.n));
            out[e] = to2(u[((long long)b * NX + x) * nz + r], T2{});
        }
    }
    if (uacc) {
        const long long nr = (long long)(ld.row_hi - ld.row_lo) * NX * B;
        for (long long e = e0; e < nr; e += stride) {
            const int r = ld.row_lo + (int)(e / ((long long)NX * B));
            const long long rem = e % ((long long)NX * B);
            const int x = (int)(rem / B), b = (int)(rem % B);
            double2 &g = uacc[((long long)(ld.s + r) * NX + x) * B + b];
            g = g + u[((long long)b * NX + x) * nz + r];
        }
    }
}

template <class T2> __global__ void k_add(T2 *dst, const T2 *__restrict__ src, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = dst[i] + src[i];
}

// local solves of layers `lays` through their inner contexts (see above); in /
// out: [L][4][NX][Bw] (null: none); vsrc: [N][B] or null; uacc: [N][B] or null.
// precise: the polarized operator, Newton potentials and reconstruction (tight
// inner tolerance), else the preconditioner (opts.inner_tol)
template <class T2>
static void nested_apply(hz_ctx *c, int B, const std::vector<int> &lays, const T2 *in, int Bw, const double2 *vsrc,
                         T2 *out, double2 *uacc, bool precise) {
    const int NX = c->NX, L = c->L;
    if (c->n_bw < Bw) {  // FP64 source / solution volumes on the transposed layer grids
        for (int l = 0; l < L; l++) {
            if (c->nsrc.size() == (size_t)L) {
                c->dfree(c->nsrc[l]);
                c->dfree(c->nsol[l]);
            }
        }
        c->nsrc.assign(L, nullptr);
        c->nsol.assign(L, nullptr);
        for (int l = 0; l < L; l++) {
            const long long n = (long long)Bw * NX * c->layers[l].nz;
            c->nsrc[l] = (double2 *)c->dalloc(sizeof(double2) * n);
            c->nsol[l] = (double2 *)c->dalloc(sizeof(double2) * n);
        }
        c->n_bw = Bw;
    }
    const long long rowsz = (long long)NX * Bw;
    for (int l : lays) {
        k_nested_src<T2><<<1024, 256, 0, c->st>>>(c->layers[l], in ? in + (long long)l * 4 * rowsz : nullptr, vsrc,
                                                  c->d_ggam, NX, Bw, B, c->p, c->nsrc[l]);
        HZ_CU(cudaGetLastError());
        c->nl++;
    }
    HZ_CU(cudaStreamSynchronize(c->st));  // the inner contexts run on their own streams
    const double tol = precise ? (c->mixed() ? 1e-6 : 1e-10) : c->opts.inner_tol;
    std::vector<hz_ctx *> ics;
    std::vector<const double2 *> fs;
    std::vector<double2 *> us;
    for (int l : lays) {
        hz_ctx *ic = Bw == B ? c->inner_ctx[l] : c->inner_wide[l];
        ic->opts.tol = tol;
        ic->nl = 0;
        ics.push_back(ic);
        fs.push_back(c->nsrc[l]);
        us.push_back(c->nsol[l]);
    }
    std::vector<hz_stats> sts;
    // an inner solve that stops at its iteration cap is still a usable inexact
    // solve (the outer FGMRES admits it); any other failure is the call's
    solve_group_impl<T2>(ics, fs, Bw, us, sts, false);
    for (const hz_stats &x : sts) c->inner_its += x.iterations;
    for (hz_ctx *ic : ics) c->nl += ic->nl;
    for (int l : lays) {
        k_nested_out<T2><<<1024, 256, 0, c->st>>>(c->layers[l], c->nsol[l], out ? out + (long long)l * 4 * rowsz : nullptr,
                                                  uacc, NX, Bw, B, c->p);
        HZ_CU(cudaGetLastError());
        c->nl++;
    }
}

template <class T2> static void nested_apply_M(hz_ctx *c, Work<T2> &W, const T2 *x, double2 *y) {
    const int B = W.B, L = c->L;
    const long long n = (long long)L * 4 * c->NX * 2 * B;
    k_stage_M<T2><<<grid1(n), 256, 0, c->st>>>(x, W.lin, L, c->NX, B);
    HZ_CU(cudaGetLastError());
    c->nl++;
    std::vector<int> all(L);
    for (int l = 0; l < L; l++) all[l] = l;
    nested_apply<T2>(c, B, all, W.lin, 2 * B, nullptr, W.lout, nullptr, true);
    const long long m = c->n_tr() * B;
    k_combine_M<T2><<<grid1(m), 256, 0, c->st>>>(x, W.lout, y, L, c->NX, B);
    HZ_CU(cudaGetLastError());
    c->nl++;
}

// the preconditioner variants of precond_inplace with every layer application an
// inner solve (B wide, inputs staged into lin, outputs added from lout)
template <class T2> static void nested_precond(hz_ctx *c, Work<T2> &W, int kind) {
    const int L = c->L, B = W.B;
    const long long rowsz = (long long)c->NX * B;
    cudaStream_t st = c->st;
    auto vrow = [&](int k, int comp) { return W.pb + ((long long)k * 4 + comp) * rowsz; };
    auto lrow = [&](T2 *base, int l, int q) { return base + ((long long)l * 4 + q) * rowsz; };
    auto cp = [&](T2 *dst, const T2 *src) {
        HZ_CU(cudaMemcpyAsync(dst, src, sizeof(T2) * rowsz, cudaMemcpyDeviceToDevice, st));
    };
    auto zero = [&](T2 *dst) { HZ_CU(cudaMemsetAsync(dst, 0, sizeof(T2) * rowsz, st)); };
    auto add = [&](T2 *dst, const T2 *src) {
        k_add<T2><<<grid1(rowsz), 256, 0, st>>>(dst, src, rowsz);
        HZ_CU(cudaGetLastError());
        c->nl++;
    };
    if (kind == 0 || kind == 1 || kind == 2) {  // d_k = v_k + G_down^k(d_{k-1})
        for (int k = 1; k <= L - 2; k++) {
            cp(lrow(W.lin, k, 0), vrow(k - 1, 0));
            cp(lrow(W.lin, k, 1), vrow(k - 1, 1));
            zero(lrow(W.lin, k, 2));
            zero(lrow(W.lin, k, 3));
            nested_apply<T2>(c, B, {k}, W.lin, B, nullptr, W.lout, nullptr, false);
            add(vrow(k, 0), lrow(W.lout, k, 2));
            add(vrow(k, 1), lrow(W.lout, k, 3));
        }
    }
    if (kind == 0 || kind == 4) {  // u-part += rows 0,1 of layer k+1 from the d-parts of interfaces k, k+1
        if (kind == 4)
            for (int k = 0; k < L - 1; k++) HZ_CU(cudaMemsetAsync(vrow(k, 2), 0, sizeof(T2) * 2 * rowsz, st));
        k_gs_fix<T2><<<grid1((long long)(L - 1) * rowsz), 256, 0, st>>>(W.pb, L - 1, c->NX, B);
        HZ_CU(cudaGetLastError());
        c->nl++;
        std::vector<int> lays;
        for (int k = 0; k < L - 1; k++) {
            const int l = k + 1;
            cp(lrow(W.lin, l, 0), vrow(k, 0));
            cp(lrow(W.lin, l, 1), vrow(k, 1));
            if (l <= L - 2) {
                cp(lrow(W.lin, l, 2), vrow(l, 0));
                cp(lrow(W.lin, l, 3), vrow(l, 1));
            } else {
                zero(lrow(W.lin, l, 2));
                zero(lrow(W.lin, l, 3));
            }
            lays.push_back(l);
        }
        nested_apply<T2>(c, B, lays, W.lin, B, nullptr, W.lout, nullptr, false);
        for (int k = 0; k < L - 1; k++) {
            add(vrow(k, 2), lrow(W.lout, k + 1, 0));
            add(vrow(k, 3), lrow(W.lout, k + 1, 1));
        }
        if (kind == 4) {
            k_refl_finish<T2><<<grid1((long long)(L - 1) * rowsz), 256, 0, st>>>(W.pb, L - 1, c->NX, B);
            HZ_CU(cudaGetLastError());
            c->nl++;
        }
    }
    if (kind == 0 || kind == 1 || kind == 3) {  // u_k = v_k + G_up^{k+1}(u_{k+1})
        for (int k = L - 3; k >= 0; k--) {
            zero(lrow(W.lin, k + 1, 0));
            zero(lrow(W.lin, k + 1, 1));
            cp(lrow(W.lin, k + 1, 2), vrow(k + 1, 2));
            cp(lrow(W.lin, k + 1, 3), vrow(k + 1, 3));
            nested_apply<T2>(c, B, {k + 1}, W.lin, B, nullptr, W.lout, nullptr, false);
            add(vrow(k, 2), lrow(W.lout, k + 1, 0));
            add(vrow(k, 3), lrow(W.lout, k + 1, 1));
        }
    }
}

// ------------------------------------------------------------ FGMRES ---
struct GmresOut {
    int iters = 0;
    double resid = 0;
};

// Flexible GMRES on the polarized system, one state per context so that
// several contexts (frequencies) can advance in lockstep on their own
// streams.  Right preconditioning stores z_j = P v_j (FGMRES); the Arnoldi
// basis, CGS2 orthogonalisation and the per-RHS Givens recurrences are FP64.
// One host synchronisation per iteration: both CGS2 passes and the norm of
// the new vector are reduced on the device and copied back together.
template <class T2> struct Fgmres {
    hz_ctx *c = nullptr;
    Work<T2> *W = nullptr;
    double tol = 0;
    int maxit = 0, kind = 0, B = 0, m = 0, nchunk = 1;
    long long n = 0, nB = 0;
    std::vector<std::vector<double2>> Hm, g, cs, sn;
    std::vector<double> beta0, res;
    std::vector<int> kb, conv, act;
    std::vector<double2> y;
    const double2 *r = nullptr;
    int total = 0, j = 0;
    bool finished = false;

    void dots(const double2 *V, long long vs, int nvec, const double2 *w, double2 *h) {
        dim3 g3(nchunk, (B + 31) / 32, nvec), blk(32, 8);
        k_dots<<<g3, blk, 0, c->st>>>(V, vs, w, n, B, nchunk, (double2 *)W->dots);
        HZ_CU(cudaGetLastError());
        c->nl++;
        k_dots_final<<<(nvec * B + 7) / 8, 256, 0, c->st>>>((double2 *)W->dots, nchunk, B, nvec, h, 0);
        HZ_CU(cudaGetLastError());
        c->nl++;
    }
    double2 *H() { return (double2 *)W->hbuf; }
    double2 *Hh() { return (double2 *)W->hhost; }

    void init(hz_ctx *c_, Work<T2> &W_, double tol_, int maxit_, int kind_) {
        c = c_;
        W = &W_;
        tol = tol_;
        maxit = maxit_;
        kind = kind_;
        B = W->B;
        m = W->restart;
        n = c->n_tr();
        nB = n * B;
        nchunk = dots_chunks(n, B);
        Hm.assign(B, std::vector<double2>((size_t)(m + 1) * m));
        g.assign(B, std::vector<double2>(m + 1));
        cs.assign(B, std::vector<double2>(m));
        sn.assign(B, std::vector<double2>(m));
        beta0.assign(B, 0.0);
        res.assign(B, 1.0);
        kb.assign(B, 0);
        conv.assign(B, 0);
        act.assign(B, 0);
        y.assign((size_t)m * B, make_double2(0, 0));
        total = 0;
        finished = false;
        HZ_CU(cudaMemsetAsync(W->x64, 0, sizeof(double2) * nB, c->st));
        dots(W->rhs64, 0, 1, W->rhs64, H());
        HZ_CU(cudaMemcpyAsync(Hh(), H(), sizeof(double2) * B, cudaMemcpyDeviceToHost, c->st));
    }
    void init_host() {  // after a sync
        for (int b = 0; b < B; b++) {
            const double n2 = Hh()[b].x;
            beta0[b] = std::sqrt(std::max(n2, 0.0));
            if (!std::isfinite(n2)) {  // a non-finite right-hand side: stop, report NaN
                conv[b] = 1;
                res[b] = NAN;
            } else if (!(beta0[b] > 0)) {
                conv[b] = 1;
                res[b] = 0;
            }
        }
        r = W->rhs64;
        bool all = true;
        for (int b = 0; b < B; b++)
            if (!conv[b]) all = false;
        finished = all;
    }
    // cycle start: ||r|| to the host
    void cycle_enqueue() {
        dots(r, 0, 1, r, H());
        HZ_CU(cudaMemcpyAsync(Hh(), H(), sizeof(double2) * B, cudaMemcpyDeviceToHost, c->st));
    }
    void cycle_host() {  // after a sync: V_0 = r / beta
        double *scale_h = W->rhost;
        for (int b = 0; b < B; b++) {
            double be = std::sqrt(std::max(Hh()[b].x, 0.0));
            act[b] = !conv[b] && be > 0;
            scale_h[b] = act[b] ? 1.0 / be : 0.0;
            std::fill(g[b].begin(), g[b].end(), make_double2(0, 0));
            g[b][0] = make_double2(be, 0);
            kb[b] = 0;
        }
        HZ_CU(cudaMemcpyAsync(W->rnorm, scale_h, sizeof(double) * B, cudaMemcpyHostToDevice, c->st));
        k_scale<<<grid1(nB), 256, 0, c->st>>>(r, W->rnorm, W->V, n, B);
        HZ_CU(cudaGetLastError());
        c->nl++;
        j = 0;
    }
    // one Arnoldi step: z_j = P v_j, w = M z_j, CGS2, ||w||; all reductions copied in one go
    void iter_enqueue() {
        cudaStream_t st = c->st;
        double2 *Vj = W->V + (long long)j * nB;
        T2 *Zj = W->Z + (long long)j * nB;
        k_cast<double2, T2><<<grid1(nB), 256, 0, st>>>(Vj, W->pb, nB);
        HZ_CU(cudaGetLastError());
        c->nl++;
        if (kind != HZ_PNONE) precond_inplace(c, *W, kind == HZ_PJAC ? 1 : 0);
        HZ_CU(cudaMemcpyAsync(Zj, W->pb, sizeof(T2) * nB, cudaMemcpyDeviceToDevice, st));
        apply_M(c, *W, Zj, W->w64);
        double2 *h1 = H(), *h2 = H() + (long long)(j + 1) * B, *nr = H() + (long long)(2 * j + 2) * B;
        dots(W->V, nB, j + 1, W->w64, h1);
        k_axpy_multi<<<grid1(nB), 256, 0, st>>>(W->V, nB, h1, j + 1, W->w64, n, B);
        HZ_CU(cudaGetLastError());
        dots(W->V, nB, j + 1, W->w64, h2);
        k_axpy_multi<<<grid1(nB), 256, 0, st>>>(W->V, nB, h2, j + 1, W->w64, n, B);
        HZ_CU(cudaGetLastError());
        c->nl += 2;
        dots(W->w64, 0, 1, W->w64, nr);
        HZ_CU(cudaMemcpyAsync(Hh(), H(), sizeof(double2) * (2 * j + 3) * B, cudaMemcpyDeviceToHost, st));
    }
    // after a sync: Givens update; returns true when the cycle ends
    bool iter_host() {
        const double2 *h1 = Hh(), *h2 = Hh() + (long long)(j + 1) * B, *nrm2 = Hh() + (long long)(2 * j + 2) * B;
        double *scale_h = W->rhost;
        total++;
        bool all = true;
        for (int b = 0; b < B; b++) {
            const double nrm = std::sqrt(std::max(nrm2[b].x, 0.0));
            scale_h[b] = 0.0;
            if (!act[b]) continue;
            auto &Hb = Hm[b];
            for (int i = 0; i <= j; i++) Hb[(size_t)i * m + j] = h1[(size_t)i * B + b] + h2[(size_t)i * B + b];
            Hb[(size_t)(j + 1) * m + j] = make_double2(nrm, 0);
            for (int i = 0; i < j; i++) {  // previous rotations [c s; -conj(s) c], c real
                double2 a = Hb[(size_t)i * m + j], bb = Hb[(size_t)(i + 1) * m + j];
                double2 csi = cs[b][i], sni = sn[b][i];
                double2 t1 = make_double2(csi.x * a.x + (sni.x * bb.x - sni.y * bb.y),
                                          csi.x * a.y + (sni.x * bb.y + sni.y * bb.x));
                double2 t2 = make_double2(-(sni.x * a.x + sni.y * a.y) + csi.x * bb.x,
                                          -(sni.x * a.y - sni.y * a.x) + csi.x * bb.y);
                Hb[(size_t)i * m + j] = t1;
                Hb[(size_t)(i + 1) * m + j] = t2;
            }
            double2 a = Hb[(size_t)j * m + j];
            double an = std::hypot(a.x, a.y);
            double den = std::hypot(an, nrm);
            double2 csj, snj;
            if (den == 0) {
                csj = make_double2(1, 0);
                snj = make_double2(0, 0);
            } else if (an == 0) {
                csj = make_double2(0, 0);
                snj = make_double2(1, 0);
            } else {
                csj = make_double2(an / den, 0);
                snj = make_double2(a.x / an * nrm / den, a.y / an * nrm / den);
            }
            cs[b][j] = csj;
            sn[b][j] = snj;
            Hb[(size_t)j * m + j] = make_double2(csj.x * a.x + snj.x * nrm, csj.x * a.y + snj.y * nrm);
            Hb[(size_t)(j + 1) * m + j] = make_double2(0, 0);
            double2 gj = g[b][j];
            g[b][j] = make_double2(csj.x * gj.x, csj.x * gj.y);
            g[b][j + 1] = make_double2(-(snj.x * gj.x + snj.y * gj.y), -(snj.x * gj.y - snj.y * gj.x));
            kb[b] = j + 1;
            res[b] = std::hypot(g[b][j + 1].x, g[b][j + 1].y) / beta0[b];
            if (!std::isfinite(res[b]) || !std::isfinite(nrm)) {  // non-finite: stop this RHS, report NaN
                res[b] = NAN;
                kb[b] = j;  // the last column holds non-finite entries
                act[b] = 0;
                conv[b] = 1;
            } else if (res[b] <= tol) {
                conv[b] = 1;
                act[b] = 0;
            } else if (nrm > 1e-300) {
                scale_h[b] = 1.0 / nrm;
            } else {  // exact breakdown: the solution is in the current space
                act[b] = 0;
                conv[b] = 1;
            }
            if (act[b]) all = false;
        }
        j++;
        const bool stop = all || total >= maxit || j >= m;
        if (!stop) {
            HZ_CU(cudaMemcpyAsync(W->rnorm, scale_h, sizeof(double) * B, cudaMemcpyHostToDevice, c->st));
            k_scale<<<grid1(nB), 256, 0, c->st>>>(W->w64, W->rnorm, W->V + (long long)j * nB, n, B);
            HZ_CU(cudaGetLastError());
            c->nl++;
        }
        return stop;
    }
    // cycle end: x += Z y; returns true when FGMRES is done, else enqueues the restart residual
    bool cycle_finish() {
        cudaStream_t st = c->st;
        std::fill(y.begin(), y.end(), make_double2(0, 0));
        for (int b = 0; b < B; b++) {
            const int k = kb[b];
            auto &Hb = Hm[b];
            std::vector<double2> yb(k);
            for (int i = k - 1; i >= 0; i--) {
                double2 sacc = g[b][i];
                for (int q = i + 1; q < k; q++) sacc = sacc - Hb[(size_t)i * m + q] * yb[q];
                yb[i] = cdiv(sacc, Hb[(size_t)i * m + i]);
            }
            for (int i = 0; i < k; i++) y[(size_t)i * B + b] = yb[i];
        }
        double2 *y_d = (double2 *)W->dots;  // reduction scratch is idle here
        HZ_CU(cudaMemcpyAsync(y_d, y.data(), sizeof(double2) * j * B, cudaMemcpyHostToDevice, st));
        k_update_x<T2><<<grid1(nB), 256, 0, st>>>(W->Z, nB, y_d, j, W->x64, n, B);
        HZ_CU(cudaGetLastError());
        c->nl++;
        bool all = true;
        for (int b = 0; b < B; b++)
            if (!conv[b]) all = false;
        if (all || total >= maxit) {
            finished = true;
            return true;
        }
        k_cast<double2, T2><<<grid1(nB), 256, 0, st>>>(W->x64, W->pa, nB);
        HZ_CU(cudaGetLastError());
        c->nl++;
        apply_M(c, *W, W->pa, W->w64);
        k_sub<<<grid1(nB), 256, 0, st>>>(W->rhs64, W->w64, W->w64, nB);
        HZ_CU(cudaGetLastError());
        c->nl++;
        r = W->w64;
        return false;
    }
    GmresOut out() const {
        GmresOut o;
        o.iters = total;
        for (int b = 0; b < B; b++) o.resid = nanmax(o.resid, res[b]);
        return o;
    }
};

static void sync_all(const std::vector<hz_ctx *> &cs);
// Bi-CGstab on the polarized system with right preconditioning (the paper's
// second Krylov method, §5): M P y = b, x = P y.  Per iteration two
// preconditioner and two operator applications; per-RHS scalars in FP64 on
// the host, three synchronisations per iteration (shared by a group).
// Vectors (FP64) live in the Krylov basis buffer: V0 = r^, V1 = r, V2 = p,
// V3 = v, V4 = s, V5 = t; P p and P s in the working precision in Z0, Z1.
template <class T2> struct Bicgstab {
    hz_ctx *c = nullptr;
    Work<T2> *W = nullptr;
    double tol = 0;
    int maxit = 0, kind = 0, B = 0, nchunk = 1, total = 0;
    long long n = 0, nB = 0;
    std::vector<double> bnorm, res;
    std::vector<double2> rho, alpha, omega;
    std::vector<int> act;
    bool finished = false;

    double2 *vec(int i) { return W->V + (long long)i * nB; }
    T2 *zv(int i) { return W->Z + (long long)i * nB; }
    double2 *H() { return (double2 *)W->hbuf; }
    double2 *Hh() { return (double2 *)W->hhost; }
    double2 *coef_d(int i) { return (double2 *)W->dots + (long long)i * B; }  // small coefficient arrays
    void dot(const double2 *a, const double2 *b, double2 *h) {
        dim3 g3(nchunk, (B + 31) / 32, 1), blk(32, 8);
        k_dots<<<g3, blk, 0, c->st>>>(a, 0, b, n, B, nchunk, (double2 *)W->dots + 8LL * B);
        HZ_CU(cudaGetLastError());
        k_dots_final<<<(B + 7) / 8, 256, 0, c->st>>>((double2 *)W->dots + 8LL * B, nchunk, B, 1, h, 0);
        HZ_CU(cudaGetLastError());
        c->nl += 2;
    }
    void precond_to(const double2 *x, T2 *z) {  // z = P x
        k_cast<double2, T2><<<grid1(nB), 256, 0, c->st>>>(x, W->pb, nB);
        HZ_CU(cudaGetLastError());
        c->nl++;
        if (kind != HZ_PNONE) precond_inplace(c, *W, kind == HZ_PJAC ? 1 : 0);
        HZ_CU(cudaMemcpyAsync(z, W->pb, sizeof(T2) * nB, cudaMemcpyDeviceToDevice, c->st));
    }
    // coefficient array -> device slot, staged in pinned memory beyond the
    // reduction results (each slot has its own staging, reused only after a sync)
    void upload(const std::vector<double2> &v, int slot) {
        double2 *hst = Hh() + 8LL * B + (long long)slot * B;
        std::copy(v.begin(), v.end(), hst);
        HZ_CU(cudaMemcpyAsync(coef_d(slot), hst, sizeof(double2) * B, cudaMemcpyHostToDevice, c->st));
    }

    void init(hz_ctx *c_, Work<T2> &W_, double tol_, int maxit_, int kind_) {
        c = c_;
        W = &W_;
        tol = tol_;
        maxit = maxit_;
        kind = kind_;
        B = W->B;
        n = c->n_tr();
        nB = n * B;
        nchunk = dots_chunks(n, B);
        bnorm.assign(B, 0.0);
        res.assign(B, 1.0);
        rho.assign(B, make_double2(1, 0));
        alpha.assign(B, make_double2(1, 0));
        omega.assign(B, make_double2(1, 0));
        act.assign(B, 1);
        total = 0;
        finished = false;
        cudaStream_t st = c->st;
        HZ_CU(cudaMemsetAsync(W->x64, 0, sizeof(double2) * nB, st));
        HZ_CU(cudaMemcpyAsync(vec(0), W->rhs64, sizeof(double2) * nB, cudaMemcpyDeviceToDevice, st));  // r^ = b
        HZ_CU(cudaMemcpyAsync(vec(1), W->rhs64, sizeof(double2) * nB, cudaMemcpyDeviceToDevice, st));  // r = b
        HZ_CU(cudaMemsetAsync(vec(2), 0, sizeof(double2) * nB, st));                                   // p = 0
        HZ_CU(cudaMemsetAsync(vec(3), 0, sizeof(double2) * nB, st));                                   // v = 0
        dot(vec(1), vec(1), H());  // ||b||^2 = <r^, r>
        HZ_CU(cudaMemcpyAsync(Hh(), H(), sizeof(double2) * B, cudaMemcpyDeviceToHost, st));
    }
    void init_host() {
        bool any = false;
        for (int b = 0; b < B; b++) {
            bnorm[b] = std::sqrt(std::max(Hh()[b].x, 0.0));
            act[b] = bnorm[b] > 0 && std::isfinite(Hh()[b].x);
            res[b] = act[b] ? 1.0 : (std::isfinite(Hh()[b].x) ? 0.0 : NAN);
            rho[b] = Hh()[b];  // <r^, r> with r^ = r = b
            any = any || act[b];
        }
        finished = !any;
    }
    // A: p = r + beta (p - omega v), v = M P p, <r^, v>
    void a_enqueue() {
        std::vector<double2> beta(B, make_double2(0, 0)), om(B, make_double2(0, 0));
        for (int b = 0; b < B; b++)
            if (act[b]) {
                beta[b] = total == 0 ? make_double2(0, 0) : cdiv(rho[b] * alpha[b], rho_prev[b] * omega[b]);
                om[b] = omega[b];
            }
        upload(beta, 0);
        upload(om, 1);
        k_bicg_p<<<grid1(nB), 256, 0, c->st>>>(vec(2), vec(1), vec(3), coef_d(0), coef_d(1), n, B);
        HZ_CU(cudaGetLastError());
        c->nl++;
        precond_to(vec(2), zv(0));
        apply_M(c, *W, zv(0), vec(3));
        dot(vec(0), vec(3), H());
        HZ_CU(cudaMemcpyAsync(Hh(), H(), sizeof(double2) * B, cudaMemcpyDeviceToHost, c->st));
    }
    std::vector<double2> rho_prev = std::vector<double2>();
    void a_host() {
        for (int b = 0; b < B; b++) {
            if (!act[b]) {
                alpha[b] = make_double2(0, 0);
                continue;
            }
            const double2 rv = Hh()[b];
            if (std::hypot(rv.x, rv.y) == 0) {  // breakdown: keep the current iterate
                act[b] = 0;
                alpha[b] = make_double2(0, 0);
                continue;
            }
            alpha[b] = cdiv(rho[b], rv);
        }
    }
    // B: s = r - alpha v, t = M P s, <t, s>, <t, t>
    void b_enqueue() {
        std::vector<double2> na(B);
        for (int b = 0; b < B; b++) na[b] = make_double2(-alpha[b].x, -alpha[b].y);
        upload(na, 2);
        k_zaxpy<<<grid1(nB), 256, 0, c->st>>>(vec(4), vec(1), vec(3), coef_d(2), n, B);
        HZ_CU(cudaGetLastError());
        c->nl++;
        precond_to(vec(4), zv(1));
        apply_M(c, *W, zv(1), vec(5));
        dot(vec(5), vec(4), H());
        dot(vec(5), vec(5), H() + B);
        HZ_CU(cudaMemcpyAsync(Hh(), H(), sizeof(double2) * 2 * B, cudaMemcpyDeviceToHost, c->st));
    }
    void b_host() {
        for (int b = 0; b < B; b++) {
            if (!act[b]) {
                omega[b] = make_double2(0, 0);
                continue;
            }
            const double tt = Hh()[B + b].x;
            omega[b] = tt > 0 ? make_double2(Hh()[b].x / tt, Hh()[b].y / tt) : make_double2(0, 0);
        }
    }
    // C: x += alpha P p + omega P s, r = s - omega t, <r^, r>, <r, r>
    void c_enqueue() {
        std::vector<double2> al(B), om(B), no(B);
        for (int b = 0; b < B; b++) {
            al[b] = act[b] ? alpha[b] : make_double2(0, 0);
            om[b] = act[b] ? omega[b] : make_double2(0, 0);
            no[b] = act[b] ? make_double2(-omega[b].x, -omega[b].y) : make_double2(0, 0);
        }
        upload(al, 3);  // slots 3, 4: coefficients of P p (Z0) and P s (Z1)
        upload(om, 4);
        upload(no, 5);
        k_update_x<T2><<<grid1(nB), 256, 0, c->st>>>(W->Z, nB, coef_d(3), 2, W->x64, n, B);
        HZ_CU(cudaGetLastError());
        k_zaxpy<<<grid1(nB), 256, 0, c->st>>>(vec(1), vec(4), vec(5), coef_d(5), n, B);
        HZ_CU(cudaGetLastError());
        c->nl += 2;
        dot(vec(0), vec(1), H());
        dot(vec(1), vec(1), H() + B);
        HZ_CU(cudaMemcpyAsync(Hh(), H(), sizeof(double2) * 2 * B, cudaMemcpyDeviceToHost, c->st));
    }
    void c_host() {
        total++;
        bool any = false;
        rho_prev = rho;
        for (int b = 0; b < B; b++) {
            if (!act[b]) continue;
            res[b] = std::sqrt(std::max(Hh()[B + b].x, 0.0)) / bnorm[b];
            rho[b] = Hh()[b];
            if (!std::isfinite(Hh()[B + b].x) || !std::isfinite(rho[b].x) || !std::isfinite(rho[b].y)) {
                res[b] = NAN;  // non-finite: stop this RHS, report NaN
                act[b] = 0;
            } else if (res[b] <= tol || std::hypot(rho[b].x, rho[b].y) == 0 ||
                std::hypot(omega[b].x, omega[b].y) == 0)
                act[b] = 0;
            any = any || act[b];
        }
        finished = !any || total >= maxit;
    }
    GmresOut out() const {
        GmresOut o;
        o.iters = total;
        for (int b = 0; b < B; b++) o.resid = nanmax(o.resid, res[b]);
        return o;
    }
};

// Lockstep Bi-CGstab over several contexts
template <class T2> static void bicgstab_group(std::vector<Bicgstab<T2> *> &gs) {
    std::vector<hz_ctx *> cs;
    for (auto *g : gs) cs.push_back(g->c);
    sync_all(cs);
    for (auto *g : gs) g->init_host();
    while (true) {
        std::vector<Bicgstab<T2> *> live;
        for (auto *g : gs)
            if (!g->finished) live.push_back(g);
        if (live.empty()) break;
        for (auto *g : live) g->a_enqueue();
        sync_all(cs);
        for (auto *g : live) g->a_host();
        for (auto *g : live) g->b_enqueue();
        sync_all(cs);
        for (auto *g : live) g->b_host();
        for (auto *g : live) g->c_enqueue();
        sync_all(cs);
        for (auto *g : live) g->c_host();
    }
}

static void sync_all(const std::vector<hz_ctx *> &cs) {
    for (hz_ctx *c : cs) HZ_CU(cudaStreamSynchronize(c->st));
}

// Lockstep FGMRES over several contexts (each on its own stream)
template <class T2> static void fgmres_group(std::vector<Fgmres<T2> *> &gs) {
    std::vector<hz_ctx *> cs;
    for (auto *g : gs) cs.push_back(g->c);
    sync_all(cs);
    for (auto *g : gs) g->init_host();
    while (true) {
        std::vector<Fgmres<T2> *> live;
        for (auto *g : gs)
            if (!g->finished) live.push_back(g);
        if (live.empty()) break;
        for (auto *g : live) g->cycle_enqueue();
        sync_all(cs);
        for (auto *g : live) g->cycle_host();
        std::vector<Fgmres<T2> *> in_cycle = live;
        while (!in_cycle.empty()) {
            for (auto *g : in_cycle) g->iter_enqueue();
            sync_all(cs);
            std::vector<Fgmres<T2> *> next;
            for (auto *g : in_cycle)
                if (!g->iter_host()) next.push_back(g);
                else g->cycle_finish();
            in_cycle.swap(next);
        }
    }
}

template <class T2>
static GmresOut fgmres(hz_ctx *c, Work<T2> &W, double tol, int maxit, int kind) {
    Fgmres<T2> g;
    g.init(c, W, tol, maxit, kind);
    std::vector<Fgmres<T2> *> gs{&g};
    fgmres_group(gs);
    return g.out();
}

// ------------------------------------------------------- nested solve ---
struct Timers {
    double local = 0, gmres = 0, recon = 0, resid = 0;
};
static double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Stage 1 of a pass of Alg. matrix_free_solver (lines 2-7) on the
// symmetric-form source src ([N][B], FP64): Newton potentials of every layer
// through cell solves and inner sweeps, sampled into the polarized
// right-hand side.
// Local solves of every cell on the symmetric-form source src ([N][B], FP64)
// into W.vol, and the inner right-hand side of every layer (W.inner_f) from them.
template <class T2> static void local_enqueue(hz_ctx *c, Work<T2> &W, const double2 *src) {
    cudaStream_t st = c->st;
    const int B = W.B, L = c->L, ncell = (int)c->cells.size();
    const int nb = (int)std::min<long long>(1024, (c->tot_vol * B / ncell + 255) / 256 + 1);
    k_scatter<T2><<<dim3(nb, ncell), 256, 0, st>>>(c->d_cells, src, W.vol, c->NX, B);
    HZ_CU(cudaGetLastError());
    c->nl++;
    cell_chain<T2>(c, W.vol, B);
    if (c->C > 1) {
        k_gather_inner<T2><<<dim3(256, L), 256, 0, st>>>(c->d_layers, c->d_cells, W.vol, W.inner_f, B, c->p);
        HZ_CU(cudaGetLastError());
        c->nl++;
    }
}

// Stage 1 of a pass of Alg. matrix_free_solver (lines 2-7) on the
// symmetric-form source src ([N][B], FP64): Newton potentials of every layer
// through cell solves and inner sweeps, sampled into the polarized
// right-hand side.
template <class T2> static void newton_enqueue(hz_ctx *c, Work<T2> &W, const double2 *src) {
    cudaStream_t st = c->st;
    const int B = W.B, L = c->L, ncell = (int)c->cells.size();
    W.cur_src = src;
    if (c->nested()) {  // every layer's Newton potential by an inner solve, sampled at rows 0, 1, n, n+1
        std::vector<int> all(L);
        for (int l = 0; l < L; l++) all[l] = l;
        nested_apply<T2>(c, B, all, (const T2 *)nullptr, B, src, W.lout, nullptr, true);
        k_pol_rhs<T2><<<grid1(c->n_tr() * B), 256, 0, st>>>(W.lout, W.rhs64, L - 1, c->NX, B);
        HZ_CU(cudaGetLastError());
        c->nl++;
        return;
    }
    local_enqueue<T2>(c, W, src);
    // keep the inner right-hand side (inner_f) for the reconstruction; solve a copy (the
    // compressed-block LU reads its right-hand sides from innerH)
    HZ_CU(cudaMemcpyAsync(c->lr_r > 0 ? W.innerH : W.inner, W.inner_f, sizeof(T2) * c->tot_inner * B,
                          cudaMemcpyDeviceToDevice, st));
    chain_layers(c, W, false, 0, L);
    k_samples<T2><<<dim3(64, ncell), 256, 0, st>>>(c->d_cells, W.vol, W.lout, c->NX, B, c->p);
    HZ_CU(cudaGetLastError());
    c->nl++;
    run(c, W.e_newton);
    k_pol_rhs<T2><<<grid1(c->n_tr() * B), 256, 0, st>>>(W.lout, W.rhs64, L - 1, c->NX, B);
    HZ_CU(cudaGetLastError());
    c->nl++;
}

// Stage 3 (lines 10-18): the volume from the traces, added to W.u.
template <class T2> static void recon_enqueue(hz_ctx *c, Work<T2> &W) {
    cudaStream_t st = c->st;
    const int B = W.B, L = c->L, ncell = (int)c->cells.size();
    const int nb = (int)std::min<long long>(1024, (c->tot_vol * B / ncell + 255) / 256 + 1);
    k_traces<T2><<<grid1((long long)(L - 1) * 2 * c->NX * B), 256, 0, st>>>(W.x64, W.pc, L - 1, c->NX, B);
    HZ_CU(cudaGetLastError());
    c->nl++;
    if (c->nested()) {  // every layer's field: source + forcing of its interface traces, owned rows into u
        const long long rowsz = (long long)c->NX * B;
        std::vector<int> all(L);
        for (int l = 0; l < L; l++) {
            all[l] = l;
            T2 *li = W.lin + (long long)l * 4 * rowsz;
            for (int q = 0; q < 4; q++) {
                const int k = q < 2 ? l - 1 : l;  // top pair: interface l-1; bottom pair: interface l
                if (k >= 0 && k < L - 1)
                    HZ_CU(cudaMemcpyAsync(li + q * rowsz, W.pc + ((long long)k * 2 + (q & 1)) * rowsz,
                                          sizeof(T2) * rowsz, cudaMemcpyDeviceToDevice, st));
                else
                    HZ_CU(cudaMemsetAsync(li + q * rowsz, 0, sizeof(T2) * rowsz, st));
            }
        }
        nested_apply<T2>(c, B, all, W.lin, B, W.cur_src, (T2 *)nullptr, W.u, true);
        return;
    }
    HZ_CU(cudaMemcpyAsync(c->lr_r > 0 ? W.innerH : W.inner, W.inner_f, sizeof(T2) * c->tot_inner * B,
                          cudaMemcpyDeviceToDevice, st));
    run(c, W.f_rec);
    chain_layers(c, W, false, 0, L);
    HZ_CU(cudaMemsetAsync(W.vol2, 0, sizeof(T2) * c->tot_vol * B, st));
    k_recon_src<T2><<<dim3(64, ncell), 256, 0, st>>>(c->d_cells, c->d_layers, W.pc, W.inner, W.vol2, L, c->NX, B, c->p,
                                                     c->d_ggam, c->d_lbeta);
    HZ_CU(cudaGetLastError());
    c->nl++;
    cell_chain<T2>(c, W.vol2, B);
    k_accum_u<T2><<<dim3(nb, ncell), 256, 0, st>>>(c->d_cells, W.vol, W.vol2, W.u, c->NX, B);
    HZ_CU(cudaGetLastError());
    c->nl++;
}

// point chunks of the residual (general batch widths)
static int residual_chunks(int) { return 256; }

// launch the residual kernel; returns the number of per-RHS partial sums written to part
// (part holds at least 4096 B + B doubles)
static int residual_launch(hz_ctx *c, const double2 *u, const double2 *fs, double2 *r, int B, int mode, double *part) {
    if (B <= 256 && (256 % B) == 0) {
        int lgB = 0;
        while ((1 << lgB) < B) lgB++;
        const int R = std::max(1, (c->NZ + 1023) / 1024), nchunk = (c->NZ + R - 1) / R;
        k_residual_rows<<<nchunk, 256, 0, c->st>>>(u, fs, r, c->d_gdiag, c->d_gcx, c->d_gcz, c->d_gD, c->NX, c->NZ,
                                                   lgB, R, part, mode);
        HZ_CU(cudaGetLastError());
        return nchunk;
    }
    const int nchunk = residual_chunks(B);
    dim3 g(nchunk, (B + 31) / 32), blk(32, 8);
    k_residual<<<g, blk, 0, c->st>>>(u, fs, r, c->d_gdiag, c->d_gcx, c->d_gcz, c->d_gD, c->NX, c->NZ, B, part,
                                     nchunk, mode);
    HZ_CU(cudaGetLastError());
    return nchunk;
}

// per-RHS ||alpha r||^2 partial sums -> host buffer (mode 0 writes r = fs - H u);
// enqueued only: valid after the stream synchronises
static void residual_enqueue(hz_ctx *c, const double2 *u, const double2 *fs, double2 *r, int B, double *out_host,
                             int mode, double *part) {
    const int nchunk = residual_launch(c, u, fs, r, B, mode, part);
    double *fin = part + (long long)nchunk * B;
    k_reduce_parts<<<(B + 255) / 256, 256, 0, c->st>>>(part, nchunk, B, fin);
    HZ_CU(cudaGetLastError());
    c->nl += 2;
    HZ_CU(cudaMemcpyAsync(out_host, fin, sizeof(double) * B, cudaMemcpyDeviceToHost, c->st));
}

static void residual_norms(hz_ctx *c, const double2 *u, const double2 *fs, double2 *r, int B, double *out_host,
                           int mode, double *part) {
    const int nchunk = residual_launch(c, u, fs, r, B, mode, part);
    double *fin = part + (long long)nchunk * B;
    k_reduce_parts<<<(B + 255) / 256, 256, 0, c->st>>>(part, nchunk, B, fin);
    HZ_CU(cudaGetLastError());
    c->nl += 2;
    HZ_CU(cudaMemcpyAsync(out_host, fin, sizeof(double) * B, cudaMemcpyDeviceToHost, c->st));
    HZ_CU(cudaStreamSynchronize(c->st));
}

// the context's device status block: error word cleared, wait limit from the options
static void init_status(hz_ctx *c) {
    c->d_err = (int *)c->dalloc(16);
    const double ms = c->opts.wait_ms > 0 ? c->opts.wait_ms : 1000.0;
    int blk[4] = {0, 0, 0, 0};
    const unsigned long long ns = (unsigned long long)(ms * 1e6);
    std::memcpy(blk + 2, &ns, sizeof ns);
    HZ_CU(cudaMemcpy(c->d_err, blk, sizeof blk, cudaMemcpyHostToDevice));
}

void init_global_alpha(hz_ctx *c) {
    init_status(c);
    c->d_ax = (double2 *)c->dalloc(sizeof(double2) * c->NX);
    c->d_axh = (double2 *)c->dalloc(sizeof(double2) * (c->NX + 1));
    c->d_az = (double2 *)c->dalloc(sizeof(double2) * c->NZ);
    c->d_azh = (double2 *)c->dalloc(sizeof(double2) * (c->NZ + 1));
    int n = std::max(c->NX, c->NZ) + 1;
    k_global_alpha<<<(n + 255) / 256, 256, 0, c->st>>>(c->NX, c->NZ, c->n_x, c->n_z, c->p, c->h, c->pml_C, c->omega,
                                                        c->d_ax, c->d_axh, c->d_az, c->d_azh);
    HZ_CU(cudaGetLastError());
    // the whole grid as one box: same coefficient kernel as the cells
    const long long N = (long long)c->NX * c->NZ;
    CellDesc g{};
    g.nx = c->NX;
    g.nz = c->NZ;
    g.w = c->n_x;
    g.n = c->n_z;
    c->d_gcell = (CellDesc *)c->dalloc(sizeof(CellDesc));
    HZ_CU(cudaMemcpy(c->d_gcell, &g, sizeof(CellDesc), cudaMemcpyHostToDevice));
    c->d_gdiag = (double2 *)c->dalloc(sizeof(double2) * N);
    c->d_gcx = (double2 *)c->dalloc(sizeof(double2) * N);
    c->d_gcz = (double2 *)c->dalloc(sizeof(double2) * N);
    c->d_gD = (double2 *)c->dalloc(sizeof(double2) * N);
    c->d_ginvD = (double2 *)c->dalloc(sizeof(double2) * N);
    c->d_ggam = (double2 *)c->dalloc(sizeof(double2) * c->NX);
    c->d_lbeta = (double2 *)c->dalloc(sizeof(double2) * std::max(c->tot_z, 1LL));
    launch_cell_coeffs(c->d_gcell, 1, c->d_m, c->NX, c->omega, c->h, c->pml_C, c->p, c->d_gdiag, c->d_gcx, c->d_gcz,
                       c->st, nullptr);
    k_global_D<<<1024, 256, 0, c->st>>>(c->d_ax, c->d_az, c->NX, N, c->d_gD, c->d_ginvD);
    HZ_CU(cudaGetLastError());
    {
        int mx = std::max(c->NX, c->max_nz);
        k_couplings<<<dim3((mx + 255) / 256, c->L + 1), 256, 0, c->st>>>(c->d_layers, c->L, c->d_ax, c->NX, c->p, c->h,
                                                                         c->pml_C, c->omega, c->d_ggam, c->d_lbeta);
        HZ_CU(cudaGetLastError());
    }
    HZ_CU(cudaStreamSynchronize(c->st));
}

// Solve of a group of contexts (one medium/frequency each, each on its own
// stream), advanced in lockstep: Newton potentials, FGMRES, reconstruction
// and the FP64 residual of every member are enqueued before the host waits,
// so members overlap on the GPU.  A single context is a group of one.
// f_dev[i], u_dev[i]: device, batch-outer [B][N].
template <class T2>
int solve_group_impl(const std::vector<hz_ctx *> &cs, const std::vector<const double2 *> &f_dev, int B,
                     const std::vector<double2 *> &u_dev, std::vector<hz_stats> &stats, bool scale_src) {
    const int G = (int)cs.size();
    for (hz_ctx *c : cs) c->group_n = G;
    std::vector<Work<T2> *> Ws(G);
    std::vector<std::vector<double>> fn(G, std::vector<double>(B)), rn(G, std::vector<double>(B));
    std::vector<Timers> tm(G);
    std::vector<int> status(G, HZ_OK), pass_done(G, 0);
    std::vector<double> prev(G, 1.0), worst(G, 0.0);
    std::vector<const double2 *> src(G);
    stats.assign(G, hz_stats{});
    const double t0 = now_ms();
    for (int i = 0; i < G; i++) {
        hz_ctx *c = cs[i];
        c->inner_its = 0;
        Ws[i] = &work<T2>(c, B);
        Work<T2> &W = *Ws[i];
        const long long N = (long long)c->NX * c->NZ;
        transpose_in(c, f_dev[i], W.gsrc, N, B, scale_src);
        HZ_CU(cudaMemsetAsync(W.u, 0, sizeof(double2) * N * B, c->st));
        residual_enqueue(c, W.u, W.gsrc, nullptr, B, W.rhost, 1, W.rnorm);
        src[i] = W.gsrc;
    }
    sync_all(cs);
    for (int i = 0; i < G; i++)
        for (int b = 0; b < B; b++) fn[i][b] = std::sqrt(Ws[i]->rhost[b]);
    const int max_pass = std::max(1, cs[0]->opts.refine_tol > 0 ? cs[0]->opts.max_refine : 1);
    std::vector<int> live(G, 1);
    for (int pass = 0; pass < max_pass; pass++) {
        std::vector<int> idx;
        for (int i = 0; i < G; i++)
            if (live[i]) idx.push_back(i);
        if (idx.empty()) break;
        std::vector<hz_ctx *> cl;
        for (int i : idx) cl.push_back(cs[i]);
        double ta = now_ms();
        for (int i : idx) newton_enqueue<T2>(cs[i], *Ws[i], src[i]);
        sync_all(cl);
        double tb = now_ms();
        const bool bicg = cs[0]->opts.krylov == HZ_BICGSTAB;
        std::vector<Fgmres<T2>> gm(bicg ? 0 : idx.size());
        std::vector<Bicgstab<T2>> bm(bicg ? idx.size() : 0);
        std::vector<double> gtol(idx.size());
        for (size_t q = 0; q < idx.size(); q++) {
            hz_ctx *c = cs[idx[q]];
            const double tol = c->opts.tol, rtol = c->opts.refine_tol;
            const int maxit = c->fault == hz_ctx::FAULT_NOCONV ? 1 : c->opts.max_it;
            double ptol = tol;
            // a pass on the residual only has to shrink it to the target, with a 10x margin
            if (pass > 0 && rtol > 0) ptol = std::min(0.1, std::max(tol, 0.1 * rtol / std::max(prev[idx[q]], 1e-300)));
            gtol[q] = ptol;
            if (c->fault == hz_ctx::FAULT_NAN) {  // injected: a NaN in the polarized right-hand side
                const double2 nan2 = make_double2(NAN, 0.0);
                HZ_CU(cudaMemcpyAsync(Ws[idx[q]]->rhs64, &nan2, sizeof nan2, cudaMemcpyHostToDevice, c->st));
                HZ_CU(cudaStreamSynchronize(c->st));
            }
            if (bicg)
                bm[q].init(c, *Ws[idx[q]], ptol, maxit, c->opts.precond);
            else
                gm[q].init(c, *Ws[idx[q]], ptol, maxit, c->opts.precond);
        }
        if (bicg) {
            std::vector<Bicgstab<T2> *> bp;
            for (auto &g : bm) bp.push_back(&g);
            bicgstab_group(bp);
        } else {
            std::vector<Fgmres<T2> *> gp;
            for (auto &g : gm) gp.push_back(&g);
            fgmres_group(gp);
        }
        double tc = now_ms();
        for (int i : idx) recon_enqueue<T2>(cs[i], *Ws[i]);
        sync_all(cl);
        double td = now_ms();
        for (int i : idx) {
            Work<T2> &W = *Ws[i];
            residual_enqueue(cs[i], W.u, W.gsrc, W.io, B, W.rhost, 0, W.rnorm);
        }
        sync_all(cl);
        double te = now_ms();
        for (size_t q = 0; q < idx.size(); q++) {
            const int i = idx[q];
            hz_ctx *c = cs[i];
            Work<T2> &W = *Ws[i];
            tm[i].local += tb - ta;
            tm[i].gmres += tc - tb;
            tm[i].recon += td - tc;
            tm[i].resid += te - td;
            GmresOut go = bicg ? bm[q].out() : gm[q].out();
            stats[i].iterations += go.iters;
            stats[i].gmres_resid = go.resid;
            stats[i].refinements = pass + 1;
            worst[i] = 0;
            for (int b = 0; b < B; b++) {
                rn[i][b] = fn[i][b] > 0 ? std::sqrt(W.rhost[b]) / fn[i][b] : 0.0;
                worst[i] = nanmax(worst[i], rn[i][b]);
            }
            const double rtol = c->opts.refine_tol;
            // a NaN compares false with everything: every convergence test is written so that it fails
            if (!(go.resid <= gtol[q]) && (!c->mixed() || std::isnan(go.resid))) status[i] = HZ_ENOTCONV;
            prev[i] = worst[i];
            if (rtol <= 0 || worst[i] <= rtol || std::isnan(worst[i]) || c->fault == hz_ctx::FAULT_NOCONV) {
                live[i] = 0;
            } else {
                src[i] = W.io;  // next pass solves for the correction from the FP64 residual
            }
        }
    }
    for (int i = 0; i < G; i++) {
        hz_ctx *c = cs[i];
        Work<T2> &W = *Ws[i];
        const double rtol = c->opts.refine_tol;
        if (rtol > 0 && !(worst[i] <= rtol)) status[i] = HZ_ENOTCONV;
        stats[i].resid = worst[i];
        transpose_out(c, W.u, u_dev[i], (long long)c->NX * c->NZ, B);
    }
    sync_all(cs);
    for (int i = 0; i < G; i++) {
        hz_ctx *c = cs[i];
        int e = 0;
        HZ_CU(cudaMemcpy(&e, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (e) {
            HZ_CU(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->st));
            throw HzError(HZ_ETIMEOUT, "an inter-CTA exchange in the inner sweep timed out; results are invalid");
        }
        stats[i].t_total_ms = now_ms() - t0;
        stats[i].inner_iterations = (int)c->inner_its;
        stats[i].compress_rank = c->lr_r;
        stats[i].t_local_ms = tm[i].local;
        stats[i].t_gmres_ms = tm[i].gmres;
        stats[i].t_recon_ms = tm[i].recon;
        stats[i].t_resid_ms = tm[i].resid;
    }
    int worst_status = HZ_OK;
    for (int i = 0; i < G; i++)
        if (status[i] != HZ_OK) worst_status = status[i];
    return worst_status;
}
template int solve_group_impl<double2>(const std::vector<hz_ctx *> &, const std::vector<const double2 *> &, int,
                                       const std::vector<double2 *> &, std::vector<hz_stats> &, bool);
template int solve_group_impl<float2>(const std::vector<hz_ctx *> &, const std::vector<const double2 *> &, int,
                                      const std::vector<double2 *> &, std::vector<hz_stats> &, bool);

// A lane of context c: shares c's decomposition, operators and split copies
// (device pointers it does not own) and owns a non-blocking stream, its error
// word and, on first use, its workspaces.
hz_ctx *make_lane(hz_ctx *c) {
    hz_ctx *s = new hz_ctx();
    s->n_x = c->n_x, s->n_z = c->n_z, s->p = c->p, s->L = c->L, s->C = c->C;
    s->omega = c->omega, s->h = c->h, s->pml_C = c->pml_C, s->NX = c->NX, s->NZ = c->NZ;
    s->opts = c->opts;
    s->rows = c->rows, s->cols = c->cols;
    s->factored = true;
    s->cells = c->cells, s->layers = c->layers;
    s->d_cells = c->d_cells, s->d_layers = c->d_layers, s->d_layer_ids = c->d_layer_ids;
    s->tot_vol = c->tot_vol, s->tot_W = c->tot_W, s->tot_F = c->tot_F, s->tot_E = c->tot_E, s->tot_S = c->tot_S;
    s->tot_K = c->tot_K, s->tot_inner = c->tot_inner, s->tot_Wi = c->tot_Wi, s->tot_P = c->tot_P;
    s->tot_V = c->tot_V, s->max_nx = c->max_nx, s->max_nz = c->max_nz, s->max_no = c->max_no;
    s->lr_r = c->lr_r, s->tot_lr = c->tot_lr, s->tot_m = c->tot_m, s->tot_ac = c->tot_ac, s->tot_lam = c->tot_lam;
    s->d_m = c->d_m, s->d_ax = c->d_ax, s->d_axh = c->d_axh, s->d_az = c->d_az, s->d_azh = c->d_azh;
    s->d_gdiag = c->d_gdiag, s->d_gcx = c->d_gcx, s->d_gcz = c->d_gcz, s->d_gD = c->d_gD;
    s->d_ginvD = c->d_ginvD, s->d_ggam = c->d_ggam, s->d_lbeta = c->d_lbeta, s->tot_z = c->tot_z;
    s->d_gcell = c->d_gcell;
    s->o64 = c->o64, s->o32 = c->o32;
    s->wtc = c->wtc;
    s->dev = c->dev;
    s->parent = c;
    HZ_CU(cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking));
    s->own_stream = true;
    init_status(s);
    return s;
}

// Full solve of one context: f (device, batch-outer [B][N]) -> u (device), stats.
// With opts.rhs_lanes = S > 1 and B a multiple of S, the right-hand sides are
// solved as S groups in lockstep, group 0 on the context, the others on lanes.
template <class T2>
int solve_impl(hz_ctx *c, const double2 *f_dev, int B, double2 *u_dev, hz_stats *st_out, bool scale_src) {
    const int S = (c->opts.rhs_lanes > 1 && B % c->opts.rhs_lanes == 0) ? c->opts.rhs_lanes : 1;
    std::vector<hz_ctx *> cs{c};
    std::vector<const double2 *> fs{f_dev};
    std::vector<double2 *> us{u_dev};
    if (S > 1) {
        while ((int)c->lanes.size() < S - 1) c->lanes.push_back(make_lane(c));
        const long long N = (long long)c->NX * c->NZ, Bs = B / S;
        HZ_CU(cudaStreamSynchronize(c->st));  // the staged inputs are complete before the lanes read them
        for (int g = 1; g < S; g++) {
            hz_ctx *s = c->lanes[g - 1];
            s->opts.time_kernels = c->opts.time_kernels;
            s->nl = 0;
            s->kt_reset();
            cs.push_back(s);
            fs.push_back(f_dev + g * Bs * N);
            us.push_back(u_dev + g * Bs * N);
        }
    }
    std::vector<hz_stats> sts;
    int r = solve_group_impl<T2>(cs, fs, B / S, us, sts, scale_src);
    for (int g = 1; g < S; g++) {  // fold the lanes' launches and kernel timings into the context
        hz_ctx *s = cs[g];
        s->kt_collect();
        c->nl += s->nl;
        for (int i = 0; i < 3; i++) {
            c->kt_launches[i] += s->kt_launches[i];
            c->kt_ms[i] += s->kt_ms[i];
            c->kt_bytes[i] += s->kt_bytes[i];
            c->kt_flops[i] += s->kt_flops[i];
        }
    }
    if (st_out) {
        int keep = st_out->gpu_launches;
        *st_out = sts[0];
        for (int g = 1; g < S; g++) {  // the worst group
            st_out->iterations = std::max(st_out->iterations, sts[g].iterations);
            st_out->refinements = std::max(st_out->refinements, sts[g].refinements);
            st_out->resid = std::max(st_out->resid, sts[g].resid);
            st_out->gmres_resid = std::max(st_out->gmres_resid, sts[g].gmres_resid);
        }
        st_out->gpu_launches = keep;
    }
    return r;
}
template int solve_impl<double2>(hz_ctx *, const double2 *, int, double2 *, hz_stats *, bool);
template int solve_impl<float2>(hz_ctx *, const double2 *, int, double2 *, hz_stats *, bool);

// ------------------------------------------------- component helpers ---
template <class T2> void comp_cell_solve(hz_ctx *c, int ci, const double2 *g_dev, int B, double2 *x_dev) {
    Work<T2> &W = work<T2>(c, B);
    Ops<T2> &o = ops<T2>(c);
    const CellDesc &cd = c->cells[ci];
    const long long npt = (long long)cd.nx * cd.nz;
    // g [B][npt] -> vol (cell slot, [npt][B])
    transpose_in(c, g_dev, W.io, npt, B, false);
    k_cast<double2, T2><<<grid1(npt * B), 256, 0, c->st>>>(W.io, W.vol + cd.vol_off * B, npt * B);
    HZ_CU(cudaGetLastError());
    c->nl++;
    cell_chain_launch<T2>(c, c->d_cells + ci, 1, W.vol, B);
    k_cast<T2, double2><<<grid1(npt * B), 256, 0, c->st>>>(W.vol + cd.vol_off * B, W.io, npt * B);
    HZ_CU(cudaGetLastError());
    HZ_CU(cudaGetLastError());
    c->nl++;
    transpose_out(c, W.io, x_dev, npt, B);
    HZ_CU(cudaStreamSynchronize(c->st));
}
template void comp_cell_solve<double2>(hz_ctx *, int, const double2 *, int, double2 *);
template void comp_cell_solve<float2>(hz_ctx *, int, const double2 *, int, double2 *);

// tr [B][4][NX] -> lin (B-wide rows of layer l) ; out [B][4][NX]
template <class T2> void comp_layer_green(hz_ctx *c, int l, const double2 *tr_dev, int mask, int B, double2 *out_dev) {
    Work<T2> &W = work<T2>(c, B);
    const long long n4 = 4LL * c->NX;
    const long long rowsz = (long long)c->NX * B;
    // [B][4*NX] -> [4*NX][B] into io, mask rows, cast into lin (layer l block)
    transpose_in(c, tr_dev, W.io, n4, B, false);
    if (!(mask & 1)) HZ_CU(cudaMemsetAsync(W.io, 0, sizeof(double2) * 2 * rowsz, c->st));
    if (!(mask & 2)) HZ_CU(cudaMemsetAsync(W.io + 2 * rowsz, 0, sizeof(double2) * 2 * rowsz, c->st));
    T2 *lin_l = W.lin + (long long)l * 4 * rowsz;
    k_cast<double2, T2><<<grid1(n4 * B), 256, 0, c->st>>>(W.io, lin_l, n4 * B);
    HZ_CU(cudaGetLastError());
    c->nl++;
    if (c->nested()) {
        nested_apply<T2>(c, B, {l}, W.lin, B, nullptr, W.lout, nullptr, true);
    } else {
        run(c, W.f_layer[l]);
        chain_layers(c, W, false, l, 1);
        run(c, W.es_layer[l]);
    }
    T2 *lout_l = W.lout + (long long)l * 4 * rowsz;
    k_cast<T2, double2><<<grid1(n4 * B), 256, 0, c->st>>>(lout_l, W.io, n4 * B);
    HZ_CU(cudaGetLastError());
    HZ_CU(cudaGetLastError());
    c->nl++;
    transpose_out(c, W.io, out_dev, n4, B);
    HZ_CU(cudaStreamSynchronize(c->st));
}
template void comp_layer_green<double2>(hz_ctx *, int, const double2 *, int, int, double2 *);
template void comp_layer_green<float2>(hz_ctx *, int, const double2 *, int, int, double2 *);

// x, y: [B][n_tr]; which: -1 apply M, 0..4 preconditioner variants
template <class T2> void comp_polar(hz_ctx *c, int which, const double2 *x_dev, int B, double2 *y_dev) {
    Work<T2> &W = work<T2>(c, B);
    const long long n = c->n_tr(), nB = n * B;
    transpose_in(c, x_dev, W.w64, n, B, false);
    if (which < 0) {
        k_cast<double2, T2><<<grid1(nB), 256, 0, c->st>>>(W.w64, W.pa, nB);
        HZ_CU(cudaGetLastError());
        c->nl++;
        apply_M(c, W, W.pa, W.x64);
    } else {
        k_cast<double2, T2><<<grid1(nB), 256, 0, c->st>>>(W.w64, W.pb, nB);
        HZ_CU(cudaGetLastError());
        c->nl++;
        precond_inplace(c, W, which);
        k_cast<T2, double2><<<grid1(nB), 256, 0, c->st>>>(W.pb, W.x64, nB);
        HZ_CU(cudaGetLastError());
        c->nl++;
    }
    transpose_out(c, W.x64, y_dev, n, B);
    HZ_CU(cudaStreamSynchronize(c->st));
}
template void comp_polar<double2>(hz_ctx *, int, const double2 *, int, double2 *);
template void comp_polar<float2>(hz_ctx *, int, const double2 *, int, double2 *);

// checkpoint of a solve: the interface traces of u ([B][N] device) -> tr ([B][K][2][NX] device)
void comp_traces(hz_ctx *c, const double2 *u_dev, int B, double2 *tr_dev) {
    const int K = c->L - 1;
    k_get_traces<<<grid1((long long)B * K * 2 * c->NX), 256, 0, c->st>>>(
        c->d_layers, u_dev, tr_dev, K, c->NX, (long long)c->NX * c->NZ, B, c->p);
    HZ_CU(cudaGetLastError());
    c->nl++;
}

// recompute u from its source and its interface traces: local solves of f,
// then the reconstruction stage of the solver with the traces given (the
// Appendix C identity; no GMRES).  f, u: [B][N]; tr: [B][K][2][NX] (device)
template <class T2> void comp_reconstruct(hz_ctx *c, const double2 *f_dev, const double2 *tr_dev, int B, double2 *u_dev) {
    Work<T2> &W = work<T2>(c, B);
    const long long N = (long long)c->NX * c->NZ;
    transpose_in(c, f_dev, W.gsrc, N, B, true);
    HZ_CU(cudaMemsetAsync(W.u, 0, sizeof(double2) * N * B, c->st));
    W.cur_src = W.gsrc;
    if (!c->nested()) local_enqueue<T2>(c, W, W.gsrc);
    k_put_traces<<<grid1(c->n_tr() * B), 256, 0, c->st>>>(tr_dev, W.x64, c->L - 1, c->NX, B);
    HZ_CU(cudaGetLastError());
    c->nl++;
    recon_enqueue<T2>(c, W);
    transpose_out(c, W.u, u_dev, N, B);
    HZ_CU(cudaStreamSynchronize(c->st));
    int e = 0;
    HZ_CU(cudaMemcpy(&e, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
        HZ_CU(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->st));
        throw HzError(HZ_ETIMEOUT, "an inter-CTA exchange in the inner sweep timed out; results are invalid");
    }
}
template void comp_reconstruct<double2>(hz_ctx *, const double2 *, const double2 *, int, double2 *);
template void comp_reconstruct<float2>(hz_ctx *, const double2 *, const double2 *, int, double2 *);

template <class T2> void comp_residual(hz_ctx *c, const double2 *u_dev, const double2 *f_dev, int B, double *res_host) {
    Work<T2> &W = work<T2>(c, B);
    const long long N = (long long)c->NX * c->NZ;
    transpose_in(c, f_dev, W.gsrc, N, B, true);
    transpose_in(c, u_dev, W.u, N, B, false);
    std::vector<double> fn(B);
    residual_norms(c, W.u, W.gsrc, nullptr, B, W.rhost, 1, W.rnorm);
    for (int b = 0; b < B; b++) fn[b] = std::sqrt(W.rhost[b]);
    residual_norms(c, W.u, W.gsrc, W.io, B, W.rhost, 0, W.rnorm);
    for (int b = 0; b < B; b++) res_host[b] = fn[b] > 0 ? std::sqrt(W.rhost[b]) / fn[b] : 0.0;
}
template void comp_residual<double2>(hz_ctx *, const double2 *, const double2 *, int, double *);
template void comp_residual<float2>(hz_ctx *, const double2 *, const double2 *, int, double *);

}  // namespace hz

// ------------------------------------------------------ kernel timers ---
cudaEvent_t hz_ctx::ev_get() {
    if (!ev_pool.empty()) {
        cudaEvent_t e = ev_pool.back();
        ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    HZ_CU(cudaEventCreate(&e));
    return e;
}
void hz_ctx::kt_begin(int cls, double bytes, double flops) {
    if (!opts.time_kernels) return;
    KT k{cls, ev_get(), ev_get(), bytes, flops};
    HZ_CU(cudaEventRecord(k.a, st));
    kt_open.push_back(k);
}
void hz_ctx::kt_end() {
    if (!opts.time_kernels || kt_open.empty()) return;
    HZ_CU(cudaEventRecord(kt_open.back().b, st));
}
void hz_ctx::kt_collect() {
    if (kt_open.empty()) return;
    HZ_CU(cudaStreamSynchronize(st));
    for (KT &k : kt_open) {
        float ms = 0;
        HZ_CU(cudaEventElapsedTime(&ms, k.a, k.b));
        kt_ms[k.cls] += ms;
        kt_launches[k.cls]++;
        kt_bytes[k.cls] += k.bytes;
        kt_flops[k.cls] += k.flops;
        ev_pool.push_back(k.a);
        ev_pool.push_back(k.b);
    }
    kt_open.clear();
}
void hz_ctx::kt_reset() {
    for (int i = 0; i < 3; i++) {
        kt_launches[i] = 0;
        kt_ms[i] = kt_bytes[i] = kt_flops[i] = 0;
    }
}
