// Generic kernels of the CUDA path:
//   * batched segmented complex GEMM (F, E, S steps of eq. (factorization))
//   * block-tridiagonal chain solves with explicitly inverted Schur blocks:
//     cell volume solves (local solves of Alg. inner_solver) and the inner
//     compressed-block LU sweeps of Section 4.2.2
//   * pivoted Gauss-Jordan inversion (offline, FP64)
#include "hz_common.cuh"

namespace hz {

// ================================================================ GEMM ===
constexpr int GBM = 64, GBN = 32, GBK = 16;

template <class T2>
__global__ void __launch_bounds__(256) k_gemm(const GemmProb<T2> *__restrict__ probs) {
    const GemmProb<T2> &P = probs[blockIdx.y];
    const int M = P.M, N = P.N;
    const int tilesM = (M + GBM - 1) / GBM, tilesN = (N + GBN - 1) / GBN;
    const int tile = blockIdx.x;
    if (tile >= tilesM * tilesN) return;
    const int m0 = (tile % tilesM) * GBM, n0 = (tile / tilesM) * GBN;
    __shared__ T2 As[GBK][GBM + 1];
    __shared__ T2 Xs[GBK][GBN];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    T2 acc[4][2];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 2; j++) acc[i][j] = czero<T2>();
    for (int pass = 0; pass < 2; pass++) {
        const T2 *A = pass ? P.A2 : P.A;
        const long long lda = pass ? P.lda2 : P.lda;
        const int K = pass ? P.K2 : P.K;
        const int xseg = pass ? P.xseg2 : P.xseg;
        const long long ldx = pass ? P.ldx2 : P.ldx;
        const T2 *const *Xp = pass ? P.X2 : P.X;
        for (int k0 = 0; k0 < K; k0 += GBK) {
#pragma unroll
            for (int q = 0; q < 4; q++) {
                int e = tid + 256 * q, mm = e / GBK, kk = e % GBK;
                int gm = m0 + mm, gk = k0 + kk;
                As[kk][mm] = (gm < M && gk < K) ? A[(long long)gm * lda + gk] : czero<T2>();
            }
#pragma unroll
            for (int q = 0; q < 2; q++) {
                int e = tid + 256 * q, kk = e / GBN, nn = e % GBN;
                int gk = k0 + kk, gn = n0 + nn;
                T2 v = czero<T2>();
                if (gk < K && gn < N) {
                    const T2 *row = Xp[gk / xseg] + (long long)(gk % xseg) * ldx;
                    v = row[gn];
                }
                Xs[kk][nn] = v;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < GBK; kk++) {
                T2 a[4], x[2];
#pragma unroll
                for (int i = 0; i < 4; i++) a[i] = As[kk][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < 2; j++) x[j] = Xs[kk][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; i++)
#pragma unroll
                    for (int j = 0; j < 2; j++) cmac(acc[i][j], a[i], x[j]);
            }
            __syncthreads();
        }
    }
    const float al = P.alpha;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        int m = m0 + ty + 16 * i;
        if (m >= M) continue;
        T2 *row = P.Y[m / P.yseg] + (long long)(m % P.yseg) * P.ldy;
#pragma unroll
        for (int j = 0; j < 2; j++) {
            int n = n0 + tx + 16 * j;
            if (n >= N) continue;
            T2 v = acc[i][j];
            v.x *= al;
            v.y *= al;
            row[n] = P.beta ? row[n] + v : v;
        }
    }
}

template <class T2>
void launch_gemm(const GemmProb<T2> *d_probs, int nprob, int max_tiles, cudaStream_t st, int *nl) {
    if (nprob <= 0 || max_tiles <= 0) return;
    dim3 grid(max_tiles, nprob);
    k_gemm<T2><<<grid, 256, 0, st>>>(d_probs);
    HZ_CU(cudaGetLastError());
    if (nl) (*nl)++;
}
template void launch_gemm<double2>(const GemmProb<double2> *, int, int, cudaStream_t, int *);
template void launch_gemm<float2>(const GemmProb<float2> *, int, int, cudaStream_t, int *);

// ========================================================= panel GEMM ===
// out(m, n) <- sum_k A[m][k] * ts[k][n] for m < M, n < NT; A row-major in
// global memory (staged through shared memory in 64 x 32 tiles), ts a
// K x NT panel in shared memory.  256 threads; each thread owns one column n
// and RPT rows of every 64-row tile.
constexpr int PK = 32;

template <class T2, int NT, class Epi>
__device__ __forceinline__ void panel_gemm(const T2 *__restrict__ A, long long lda, int M, int K,
                                           const T2 *ts, T2 *As, Epi epi) {
    constexpr int TPC = 256 / NT;
    constexpr int RPT = 64 / TPC;
    const int tid = threadIdx.x, n = tid % NT, r0 = tid / NT;
    for (int m0 = 0; m0 < M; m0 += 64) {
        T2 acc[RPT];
#pragma unroll
        for (int r = 0; r < RPT; r++) acc[r] = czero<T2>();
        for (int k0 = 0; k0 < K; k0 += PK) {
            for (int e = tid; e < 64 * PK; e += 256) {
                int mm = e / PK, kk = e % PK;
                int gm = m0 + mm, gk = k0 + kk;
                As[mm * (PK + 1) + kk] = (gm < M && gk < K) ? A[(long long)gm * lda + gk] : czero<T2>();
            }
            __syncthreads();
            const int kmax = min(PK, K - k0);
            for (int kk = 0; kk < kmax; kk++) {
                T2 tv = ts[(k0 + kk) * NT + n];
#pragma unroll
                for (int r = 0; r < RPT; r++) cmac(acc[r], As[(r0 + TPC * r) * (PK + 1) + kk], tv);
            }
            __syncthreads();
        }
#pragma unroll
        for (int r = 0; r < RPT; r++) {
            int m = m0 + r0 + TPC * r;
            if (m < M) epi(m, n, acc[r]);
        }
    }
}

// ========================================================= cell chain ===
// Solve H^{l,c} x = g for every cell and RHS tile.  H^{l,c} is block
// tridiagonal over grid rows with diagonal couplings cz between rows; with
// W_j the inverse of the j-th Schur complement:
//   y_0 = W_0 g_0,  y_j = W_j (g_j - cz_{j-1} . y_{j-1})
//   x_{nz-1} = y_{nz-1},  x_j = y_j - W_j (cz_j . x_{j+1})
// vol layout: [cell vol_off + jz*nx + jx][B] (RHS innermost), in place.
template <class T2, int NT>
__global__ void __launch_bounds__(256) k_cell_chain(const CellDesc *__restrict__ cells, const T2 *__restrict__ W,
                                                    const T2 *__restrict__ cz, T2 *vol, int B) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const CellDesc &cd = cells[blockIdx.y];
    const int nx = cd.nx, nz = cd.nz;
    const int n0 = blockIdx.x * NT;
    if (n0 >= B) return;
    T2 *tb = reinterpret_cast<T2 *>(smraw);
    T2 *pb = tb + nx * NT;
    T2 *As = pb + nx * NT;
    const T2 *Wc = W + cd.w_off;
    const T2 *czc = cz + cd.cz_off;
    T2 *v = vol + cd.vol_off * (long long)B;
    const int tid = threadIdx.x;
    const long long rs = (long long)nx * B;
    for (int jz = 0; jz < nz; jz++) {
        T2 *g = v + jz * rs;
        for (int e = tid; e < nx * NT; e += 256) {
            int jx = e / NT, nn = e % NT;
            T2 val = czero<T2>();
            if (n0 + nn < B) {
                val = g[(long long)jx * B + n0 + nn];
                if (jz > 0) val = val - czc[(long long)(jz - 1) * nx + jx] * pb[e];
            }
            tb[e] = val;
        }
        __syncthreads();
        panel_gemm<T2, NT>(Wc + (long long)jz * nx * nx, nx, nx, nx, tb, As, [&](int m, int nn, T2 a) {
            pb[m * NT + nn] = a;
            if (n0 + nn < B) g[(long long)m * B + n0 + nn] = a;
        });
        __syncthreads();
    }
    for (int jz = nz - 2; jz >= 0; jz--) {
        for (int e = tid; e < nx * NT; e += 256) {
            int jx = e / NT;
            tb[e] = czc[(long long)jz * nx + jx] * pb[e];
        }
        __syncthreads();
        T2 *y = v + jz * rs;
        panel_gemm<T2, NT>(Wc + (long long)jz * nx * nx, nx, nx, nx, tb, As, [&](int m, int nn, T2 a) {
            T2 x = czero<T2>();
            if (n0 + nn < B) {
                x = y[(long long)m * B + n0 + nn] - a;
                y[(long long)m * B + n0 + nn] = x;
            }
            pb[m * NT + nn] = x;
        });
        __syncthreads();
    }
}

template <class T2, int NT>
static void cell_chain_nt(const CellDesc *d_cells, int ncell, const T2 *W, const T2 *cz, T2 *vol, int B, int max_nx,
                          cudaStream_t st) {
    size_t sm = (size_t)(2 * max_nx * NT + 64 * (PK + 1)) * sizeof(T2);
    HZ_CU(cudaFuncSetAttribute(k_cell_chain<T2, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    dim3 grid((B + NT - 1) / NT, ncell);
    k_cell_chain<T2, NT><<<grid, 256, sm, st>>>(d_cells, W, cz, vol, B);
    HZ_CU(cudaGetLastError());
}

template <class T2>
void launch_cell_chain(const CellDesc *d_cells, int ncell, const T2 *W, const T2 *cz, T2 *vol, int B, int max_nx,
                       cudaStream_t st, int *nl) {
    if (ncell <= 0 || B <= 0) return;
    // enough CTAs to fill the GPU: wide tiles when there are many cells
    if ((long long)ncell * ((B + 15) / 16) >= 148 || B <= 4)
        cell_chain_nt<T2, 16>(d_cells, ncell, W, cz, vol, B, max_nx, st);
    else
        cell_chain_nt<T2, 4>(d_cells, ncell, W, cz, vol, B, max_nx, st);
    if (nl) (*nl)++;
}
template void launch_cell_chain<double2>(const CellDesc *, int, const double2 *, const double2 *, double2 *, int,
                                         int, cudaStream_t, int *);
template void launch_cell_chain<float2>(const CellDesc *, int, const float2 *, const float2 *, float2 *, int, int,
                                        cudaStream_t, int *);

// ======================================================== inner chain ===
// Block LU sweeps of a layer's inner SIE (Section 4.2.2).  Interface vectors
// x_j (2 nz: a-column then b-column traces) live in slots j+1 of the layer's
// inner buffer [(C+1) * 2nz][B]; on entry slot j+1 holds the right-hand side.
//   forward : t = g_j (+ Z_j y_{j-1} on the a-half), y_j = W_j t
//   backward: x_j = y_j + V_j x_{j+1}
template <class T2, int NT>
__global__ void __launch_bounds__(256) k_inner_chain(const LayerDesc *__restrict__ layers,
                                                     const int *__restrict__ ids, const T2 *__restrict__ W,
                                                     const T2 *__restrict__ Z, const T2 *__restrict__ V, T2 *inner,
                                                     int B) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const LayerDesc &ld = layers[ids[blockIdx.y]];
    const int nz = ld.nz, n2 = 2 * nz, J = ld.C - 1;
    const int n0 = blockIdx.x * NT;
    if (J <= 0 || n0 >= B) return;
    T2 *tb = reinterpret_cast<T2 *>(smraw);
    T2 *pb = tb + n2 * NT;
    T2 *As = pb + n2 * NT;
    T2 *iv = inner + ld.inner_off * (long long)B;
    const int tid = threadIdx.x;
    const long long slot = (long long)n2 * B;
    for (int j = 0; j < J; j++) {
        T2 *g = iv + (j + 1) * slot;
        for (int e = tid; e < n2 * NT; e += 256) {
            int m = e / NT, nn = e % NT;
            tb[e] = (n0 + nn < B) ? g[(long long)m * B + n0 + nn] : czero<T2>();
        }
        __syncthreads();
        if (j > 0) {
            panel_gemm<T2, NT>(Z + ld.Z_off + (long long)j * nz * n2, n2, nz, n2, pb, As,
                               [&](int m, int nn, T2 a) { tb[m * NT + nn] = tb[m * NT + nn] + a; });
            __syncthreads();
        }
        panel_gemm<T2, NT>(W + ld.W_off + (long long)j * n2 * n2, n2, n2, n2, tb, As, [&](int m, int nn, T2 a) {
            pb[m * NT + nn] = a;
            if (n0 + nn < B) g[(long long)m * B + n0 + nn] = a;
        });
        __syncthreads();
    }
    for (int j = J - 2; j >= 0; j--) {
        T2 *y = iv + (j + 1) * slot;
        panel_gemm<T2, NT>(V + ld.V_off + (long long)j * n2 * n2, n2, n2, n2, pb, As, [&](int m, int nn, T2 a) {
            T2 x = czero<T2>();
            if (n0 + nn < B) {
                x = y[(long long)m * B + n0 + nn] + a;
                y[(long long)m * B + n0 + nn] = x;
            }
            tb[m * NT + nn] = x;
        });
        __syncthreads();
        T2 *tmp = tb;
        tb = pb;
        pb = tmp;
    }
}

template <class T2, int NT>
static void inner_chain_nt(const LayerDesc *d_layers, const int *ids, int nlayer, const T2 *W, const T2 *Z,
                           const T2 *V, T2 *inner, int B, int max_nz2, cudaStream_t st) {
    size_t sm = (size_t)(2 * max_nz2 * NT + 64 * (PK + 1)) * sizeof(T2);
    HZ_CU(cudaFuncSetAttribute(k_inner_chain<T2, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    dim3 grid((B + NT - 1) / NT, nlayer);
    k_inner_chain<T2, NT><<<grid, 256, sm, st>>>(d_layers, ids, W, Z, V, inner, B);
    HZ_CU(cudaGetLastError());
}

template <class T2>
void launch_inner_chain(const LayerDesc *d_layers, const int *d_ids, int nlayer, const T2 *W, const T2 *Z,
                        const T2 *V, T2 *inner, int B, int max_nz2, cudaStream_t st, int *nl) {
    if (nlayer <= 0 || B <= 0) return;
    if ((long long)nlayer * ((B + 15) / 16) >= 64 || B <= 4)
        inner_chain_nt<T2, 16>(d_layers, d_ids, nlayer, W, Z, V, inner, B, max_nz2, st);
    else
        inner_chain_nt<T2, 4>(d_layers, d_ids, nlayer, W, Z, V, inner, B, max_nz2, st);
    if (nl) (*nl)++;
}
template void launch_inner_chain<double2>(const LayerDesc *, const int *, int, const double2 *, const double2 *,
                                          const double2 *, double2 *, int, int, cudaStream_t, int *);
template void launch_inner_chain<float2>(const LayerDesc *, const int *, int, const float2 *, const float2 *,
                                         const float2 *, float2 *, int, int, cudaStream_t, int *);

// ============================================== offline: coefficients ===
// PML stretching alpha = 1/(1 + i sigma/omega), sigma(d) = (C/delta)(d/delta)^2
// with d the distance past the interior interval [0, (nint+1) h] of a box
// with nint interior nodes and p PML nodes (Appendix A).  k is the node
// number (half-integers for staggered positions).
__device__ inline double2 pml_alpha(double k, int nint, int p, double h, double C, double omega) {
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

// Row-scaled (complex-symmetric) 5-point operator of a cell box: the Appendix A
// rows divided by alpha_x(p) alpha_z(q):
//   coupling to (jz, jx+1): -alpha_x(s+1/2) / (alpha_z(r) h^2)
//   coupling to (jz+1, jx): -alpha_z(r+1/2) / (alpha_x(s) h^2)
//   diagonal: (alpha_x(s+1/2)+alpha_x(s-1/2))/(alpha_z h^2)
//           + (alpha_z(r+1/2)+alpha_z(r-1/2))/(alpha_x h^2) - omega^2 m/(alpha_x alpha_z)
// The cell's medium is the global m with the layer rows and cell columns
// extended into the cell's own PML by their boundary values.
__global__ void k_cell_coeffs(const CellDesc *__restrict__ cells, const double *__restrict__ m, int NX, double omega,
                              double h, double C, int p, double2 *diag, double2 *cx, double2 *cz) {
    const CellDesc &cd = cells[blockIdx.y];
    const int nx = cd.nx, nz = cd.nz;
    const double h2 = h * h;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nx * nz; e += gridDim.x * blockDim.x) {
        int jz = e / nx, jx = e % nx;
        double r = jz - p + 1.0, s = jx - p + 1.0;
        int gz = cd.s + jz, gx = cd.t + jx;
        if (cd.top) gz = max(gz, cd.s + p);
        if (cd.bot) gz = min(gz, cd.s + cd.n + p - 1);
        if (cd.left) gx = max(gx, cd.t + p);
        if (cd.right) gx = min(gx, cd.t + cd.w + p - 1);
        double mm = m[(long long)gz * NX + gx];
        double2 axc = pml_alpha(s, cd.w, p, h, C, omega), axp = pml_alpha(s + 0.5, cd.w, p, h, C, omega),
                axm = pml_alpha(s - 0.5, cd.w, p, h, C, omega);
        double2 azc = pml_alpha(r, cd.n, p, h, C, omega), azp = pml_alpha(r + 0.5, cd.n, p, h, C, omega),
                azm = pml_alpha(r - 0.5, cd.n, p, h, C, omega);
        double2 azh2 = h2 * azc, axh2 = h2 * axc;
        double2 d = cdiv(axp + axm, azh2) + cdiv(azp + azm, axh2) - cdiv(make_double2(omega * omega * mm, 0.0), axc * azc);
        long long o = cd.vol_off + e;
        diag[o] = d;
        double2 vx = cdiv(axp, azh2), vz = cdiv(azp, axh2);
        cx[o] = make_double2(-vx.x, -vx.y);
        cz[o] = make_double2(-vz.x, -vz.y);
    }
}

void launch_cell_coeffs(const CellDesc *d_cells, int ncell, const double *m, int NX, double omega, double h, double C,
                        int p, double2 *diag, double2 *cx, double2 *cz, cudaStream_t st, int *nl) {
    dim3 grid(64, ncell);
    k_cell_coeffs<<<grid, 256, 0, st>>>(d_cells, m, NX, omega, h, C, p, diag, cx, cz);
    HZ_CU(cudaGetLastError());
    if (nl) (*nl)++;
}

// ========================================= offline: Gauss-Jordan (FP64) ===
// In-place inverse of the n x n matrix A (row stride lda) by Gauss-Jordan
// elimination with partial pivoting (row exchanges, undone on the columns at
// the end).  Returns 0, or k+1 if column k has no nonzero pivot.
// Shared scratch: rowk[n], colk[n], perm[n], redv[8], redi[8].
__device__ int gj_inverse(double2 *A, int n, long long lda, double2 *rowk, double2 *colk, int *perm, double *redv,
                          int *redi) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    __shared__ int s_piv;
    __shared__ double s_best;
    for (int k = 0; k < n; k++) {
        double best = -1.0;
        int bi = k;
        for (int i = k + tid; i < n; i += blockDim.x) {
            double a = cabs2(A[(long long)i * lda + k]);
            if (a > best) {
                best = a;
                bi = i;
            }
        }
        for (int off = 16; off > 0; off >>= 1) {
            double ob = __shfl_down_sync(0xffffffffu, best, off);
            int oi = __shfl_down_sync(0xffffffffu, bi, off);
            if (ob > best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
        if (lane == 0) {
            redv[wid] = best;
            redi[wid] = bi;
        }
        __syncthreads();
        if (tid == 0) {
            double b = redv[0];
            int ii = redi[0];
            for (int w = 1; w < nw; w++)
                if (redv[w] > b || (redv[w] == b && redi[w] < ii)) {
                    b = redv[w];
                    ii = redi[w];
                }
            s_piv = ii;
            s_best = b;
            perm[k] = ii;
        }
        __syncthreads();
        if (!(s_best > 0.0)) return k + 1;
        const int pr = s_piv;
        if (pr != k)
            for (int j = tid; j < n; j += blockDim.x) {
                double2 t = A[(long long)k * lda + j];
                A[(long long)k * lda + j] = A[(long long)pr * lda + j];
                A[(long long)pr * lda + j] = t;
            }
        __syncthreads();
        const double2 inv = cdiv(make_double2(1.0, 0.0), A[(long long)k * lda + k]);
        for (int j = tid; j < n; j += blockDim.x) rowk[j] = (j == k) ? inv : A[(long long)k * lda + j] * inv;
        for (int i = tid; i < n; i += blockDim.x) colk[i] = A[(long long)i * lda + k];
        __syncthreads();
        for (int e = tid; e < n * n; e += blockDim.x) {
            int i = e / n, j = e % n;
            double2 *a = &A[(long long)i * lda + j];
            if (i == k) {
                *a = rowk[j];
            } else {
                double2 base = (j == k) ? make_double2(0.0, 0.0) : *a;
                *a = base - colk[i] * rowk[j];
            }
        }
        __syncthreads();
    }
    for (int k = n - 1; k >= 0; k--) {
        int pr = perm[k];
        if (pr != k)
            for (int i = tid; i < n; i += blockDim.x) {
                double2 t = A[(long long)i * lda + k];
                A[(long long)i * lda + k] = A[(long long)i * lda + pr];
                A[(long long)i * lda + pr] = t;
            }
        __syncthreads();
    }
    return 0;
}

__global__ void __launch_bounds__(256) k_gj(double2 *const *mats, const int *ns, int *info) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int n = ns[blockIdx.x];
    double2 *rowk = reinterpret_cast<double2 *>(smraw);
    double2 *colk = rowk + n;
    int *perm = reinterpret_cast<int *>(colk + n);
    __shared__ double redv[32];
    __shared__ int redi[32];
    int r = gj_inverse(mats[blockIdx.x], n, n, rowk, colk, perm, redv, redi);
    if (threadIdx.x == 0 && r) atomicCAS(info, 0, r);
}

void launch_gj_inverse(double2 *const *d_mats, const int *d_n, int nmat, int max_n, int *d_info, cudaStream_t st,
                       int *nl) {
    if (nmat <= 0) return;
    size_t sm = (size_t)max_n * (2 * sizeof(double2) + sizeof(int));
    HZ_CU(cudaFuncSetAttribute(k_gj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_gj<<<nmat, 256, sm, st>>>(d_mats, d_n, d_info);
    HZ_CU(cudaGetLastError());
    if (nl) (*nl)++;
}

// Cell block-tridiagonal factorization: S_0 = A_0, S_j = A_j - cz_{j-1} W_{j-1} cz_{j-1},
// W_j = S_j^{-1}, with A_j the tridiagonal x-operator of grid row j.
__global__ void __launch_bounds__(256) k_cell_factor(const CellDesc *__restrict__ cells, const double2 *diag,
                                                     const double2 *cxv, const double2 *czv, double2 *W, int *info) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const CellDesc &cd = cells[blockIdx.x];
    const int nx = cd.nx, nz = cd.nz;
    double2 *rowk = reinterpret_cast<double2 *>(smraw);
    double2 *colk = rowk + nx;
    int *perm = reinterpret_cast<int *>(colk + nx);
    __shared__ double redv[32];
    __shared__ int redi[32];
    const long long nn = (long long)nx * nx;
    for (int jz = 0; jz < nz; jz++) {
        double2 *S = W + cd.w_off + jz * nn;
        const double2 *Wp = S - nn;
        const long long o = cd.vol_off + (long long)jz * nx;
        for (int e = threadIdx.x; e < nx * nx; e += blockDim.x) {
            int i = e / nx, k = e % nx;
            double2 a = make_double2(0.0, 0.0);
            if (k == i)
                a = diag[o + i];
            else if (k == i + 1)
                a = cxv[o + i];
            else if (k == i - 1)
                a = cxv[o + k];
            if (jz > 0) {
                const double2 c1 = czv[o - nx + i], c2 = czv[o - nx + k];
                a = a - (c1 * Wp[e]) * c2;
            }
            S[e] = a;
        }
        __syncthreads();
        int r = gj_inverse(S, nx, nx, rowk, colk, perm, redv, redi);
        if (r) {
            if (threadIdx.x == 0) atomicCAS(info, 0, (blockIdx.x + 1));
            return;
        }
        __syncthreads();
    }
}

void launch_cell_factor(const CellDesc *d_cells, int ncell, const double2 *diag, const double2 *cx, const double2 *cz,
                        double2 *W, int max_nx, int *d_info, cudaStream_t st, int *nl) {
    size_t sm = (size_t)max_nx * (2 * sizeof(double2) + sizeof(int));
    HZ_CU(cudaFuncSetAttribute(k_cell_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_cell_factor<<<ncell, 256, sm, st>>>(d_cells, diag, cx, cz, W, d_info);
    HZ_CU(cudaGetLastError());
    if (nl) (*nl)++;
}

}  // namespace hz
