// Offline stage (Section 4.3.1): decomposition descriptors, per-cell
// block-tridiagonal factorization, cell Green's blocks (the dense blocks of
// M_f and M_u in eq. (factorization), split here into F, E and S), and the
// block LU of every layer's inner SIE (Section 4.2.2) with inverted diagonal
// blocks.  Everything runs on the device in FP64.
#include <algorithm>
#include <cstring>

#include "hz_ctx.cuh"

void *hz_ctx::dalloc(size_t bytes) {
    void *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (fault == FAULT_ALLOC && ++n_dalloc == fault_n) {
        char b[160];
        snprintf(b, sizeof b, "device allocation of %.3f GB failed (injected by HZ_FAULT=alloc)", bytes / 1e9);
        throw hz::HzError(HZ_ENOMEM, b);
    }
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        char b[160];
        snprintf(b, sizeof b, "device allocation of %.3f GB failed (%s)", bytes / 1e9, cudaGetErrorString(e));
        throw hz::HzError(HZ_ENOMEM, b);
    }
    allocs[p] = bytes;
    dev_bytes += (long long)bytes;
    return p;
}

void hz_ctx::dfree(void *p) {
    if (!p) return;
    auto it = allocs.find(p);
    if (it != allocs.end()) {
        dev_bytes -= (long long)it->second;
        allocs.erase(it);
    }
    cudaFree(p);
}

namespace hz {

// ------------------------------------------------ decomposition tables ---
void build_decomposition(hz_ctx *c) {
    const int p = c->p, L = c->L, C = c->C;
    c->cells.clear();
    c->layers.clear();
    c->tot_z = 0;
    long long vol = 0, Wc = 0, F = 0, E = 0, S = 0, K = 0, inner = 0, Wi = 0, Pi = 0, V = 0;
    int s = 0;
    c->max_nx = c->max_nz = c->max_no = 0;
    for (int l = 0; l < L; l++) {
        LayerDesc ld{};
        ld.n = c->rows[l];
        ld.nz = ld.n + 2 * p;
        ld.s = s;
        ld.C = C;
        ld.row_lo = (l == 0) ? 0 : p;
        ld.row_hi = (l == L - 1) ? ld.n + 2 * p : ld.n + p;
        ld.cell0 = (int)c->cells.size();
        ld.zoff = c->tot_z;
        c->tot_z += ld.n + 2 * p;
        ld.inner_off = inner;
        inner += (long long)(C + 1) * 2 * ld.nz;
        const long long n2 = 2LL * ld.nz;
        ld.W_off = Wi;
        Wi += (long long)std::max(C - 1, 0) * n2 * n2;
        ld.P_off = Pi;
        Pi += (long long)std::max(C - 1, 0) * n2 * n2;
        ld.V_off = V;
        V += (long long)std::max(C - 1, 0) * n2 * n2;
        int t = 0;
        for (int cc = 0; cc < C; cc++) {
            CellDesc cd{};
            cd.l = l;
            cd.c = cc;
            cd.top = l > 0;
            cd.bot = l < L - 1;
            cd.left = cc > 0;
            cd.right = cc < C - 1;
            cd.w = c->cols[cc];
            cd.n = ld.n;
            cd.nx = cd.w + 2 * p;
            cd.nz = ld.nz;
            cd.t = t;
            cd.s = s;
            cd.own_lo = (cc == 0) ? 0 : p;
            int own_hi = (cc == C - 1) ? cd.w + 2 * p : cd.w + p;
            cd.no = own_hi - cd.own_lo;
            cd.row_lo = ld.row_lo;
            cd.row_hi = ld.row_hi;
            cd.vol_off = vol;
            cd.cz_off = vol;
            vol += (long long)cd.nx * cd.nz;
            cd.w_off = Wc;
            cd.ldw = (cd.nx + 1) & ~1;
            Wc += (long long)cd.nz * cd.nx * cd.ldw;
            cd.F_off = F;
            F += 2LL * cd.nz * 4 * cd.no;
            cd.E_off = E;
            E += 4LL * cd.no * 4 * cd.nz;
            cd.S_off = S;
            S += 4LL * cd.no * 4 * cd.no;
            cd.K_off = K;
            K += 2LL * cd.nz * 4 * cd.nz;
            c->max_nx = std::max(c->max_nx, cd.nx);
            c->max_no = std::max(c->max_no, cd.no);
            c->cells.push_back(cd);
            t += cd.w;
        }
        c->max_nz = std::max(c->max_nz, ld.nz);
        c->layers.push_back(ld);
        s += ld.n;
    }
    c->tot_vol = vol;
    c->tot_W = Wc;
    c->tot_F = F;
    c->tot_E = E;
    c->tot_S = S;
    c->tot_K = K;
    c->tot_inner = inner;
    c->tot_Wi = Wi;
    c->tot_P = Pi;
    c->tot_V = V;
    c->d_cells = (CellDesc *)c->dalloc(sizeof(CellDesc) * c->cells.size());
    c->d_layers = (LayerDesc *)c->dalloc(sizeof(LayerDesc) * c->layers.size());
    c->d_layer_ids = (int *)c->dalloc(sizeof(int) * L);
    std::vector<int> ids(L);
    for (int l = 0; l < L; l++) ids[l] = l;
    HZ_CU(cudaMemcpy(c->d_cells, c->cells.data(), sizeof(CellDesc) * c->cells.size(), cudaMemcpyHostToDevice));
    HZ_CU(cudaMemcpy(c->d_layers, c->layers.data(), sizeof(LayerDesc) * L, cudaMemcpyHostToDevice));
    HZ_CU(cudaMemcpy(c->d_layer_ids, ids.data(), sizeof(int) * L, cudaMemcpyHostToDevice));
}

// ----------------------------------------------------- helper kernels ---
__device__ inline double2 pml_alpha_f(double k, int nint, int p, double h, double C, double omega) {
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

// Node and trace-row bookkeeping (array indices in the cell box):
//   column sources (inner interface forcing): nodes 0, 1, w, w+1
//   row sources / samples (outer interface forcing): nodes 0, 1, n, n+1
__device__ inline int col_node(const CellDesc &cd, int q, int p) {
    return q == 0 ? p - 1 : (q == 1 ? p : (q == 2 ? p + cd.w - 1 : p + cd.w));
}
__device__ inline int row_node(const CellDesc &cd, int q, int p) {
    return q == 0 ? p - 1 : (q == 1 ? p : (q == 2 ? p + cd.n - 1 : p + cd.n));
}

// Unit sources: RHS b < 4nz -> column source q = b / nz at row b % nz;
// b >= 4nz -> row source q = (b-4nz) / no at owned column (b-4nz) % no.
__global__ void k_unit_sources(const CellDesc *__restrict__ cells, double2 *X, int Bg, int p) {
    const CellDesc &cd = cells[blockIdx.y];
    const int nb = 4 * cd.nz + 4 * cd.no;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        int jz, jx;
        if (b < 4 * cd.nz) {
            jz = b % cd.nz;
            jx = col_node(cd, b / cd.nz, p);
        } else {
            int bb = b - 4 * cd.nz;
            jz = row_node(cd, bb / cd.no, p);
            jx = cd.own_lo + bb % cd.no;
        }
        X[(cd.vol_off + (long long)jz * cd.nx + jx) * Bg + b] = make_double2(1.0, 0.0);
    }
}

// Inputs of the K/E operators: i = 0..3 <-> (x_{c-1,a}, x_{c-1,b}, x_{c,a}, x_{c,b});
// the Appendix C forcing puts -beta x_{c-1,a} on column node 1, +beta x_{c-1,b}
// on node 0, +beta x_{c,a} on node w+1 and -beta x_{c,b} on node w.
__device__ inline int k_src(int i) { return i == 0 ? 1 : (i == 1 ? 0 : (i == 2 ? 3 : 2)); }
__device__ inline double k_sgn(int i) { return (i == 0 || i == 3) ? -1.0 : 1.0; }

// Extract K, F, E, S of one group of cells from the Green's solutions X
// (the group's descriptors carry vol_off relative to X; the global operator
// offsets are unchanged).
__global__ void k_extract(const CellDesc *__restrict__ cells, const double2 *__restrict__ X, int Bg, int p,
                          double h, double Cp, double omega, double2 *K, double2 *F, double2 *E, double2 *S) {
    const CellDesc &cd = cells[blockIdx.y];
    const int nz = cd.nz, no = cd.no, nx = cd.nx;
    const long long nK = 2LL * nz * 4 * nz, nF = 2LL * nz * 4 * no, nE = 4LL * no * 4 * nz, nS = 4LL * no * 4 * no;
    const long long tot = nK + nF + nE + nS;
    const double h2 = h * h;
    auto Xat = [&](int jz, int jx, int b) { return X[(cd.vol_off + (long long)jz * nx + jx) * Bg + b]; };
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        if (e < nK) {
            int row = (int)(e / (4 * nz)), col = (int)(e % (4 * nz));
            int t = row / nz, jz = row % nz, i = col / nz, jz2 = col % nz;
            double2 az = pml_alpha_f(jz2 - p + 1.0, cd.n, p, h, Cp, omega);
            double2 beta = cdiv(make_double2(-1.0, 0.0), h2 * az);
            double2 g = Xat(jz, col_node(cd, t == 0 ? 1 : 2, p), k_src(i) * nz + jz2);
            K[cd.K_off + e] = k_sgn(i) * (g * beta);
        } else if (e < nK + nF) {
            long long f = e - nK;
            int row = (int)(f / (4 * no)), col = (int)(f % (4 * no));
            int t = row / nz, jz = row % nz, i = col / no, o = col % no;
            double2 ax = pml_alpha_f(cd.own_lo + o - p + 1.0, cd.w, p, h, Cp, omega);
            double2 gam = cdiv(make_double2(-1.0, 0.0), h2 * ax);
            double2 g = Xat(jz, col_node(cd, t == 0 ? 1 : 2, p), 4 * nz + k_src(i) * no + o);
            F[cd.F_off + f] = k_sgn(i) * (g * gam);
        } else if (e < nK + nF + nE) {
            long long f = e - nK - nF;
            int row = (int)(f / (4 * nz)), col = (int)(f % (4 * nz));
            int rho = row / no, o = row % no, i = col / nz, jz2 = col % nz;
            double2 az = pml_alpha_f(jz2 - p + 1.0, cd.n, p, h, Cp, omega);
            double2 beta = cdiv(make_double2(-1.0, 0.0), h2 * az);
            double2 g = Xat(row_node(cd, rho, p), cd.own_lo + o, k_src(i) * nz + jz2);
            E[cd.E_off + f] = k_sgn(i) * (g * beta);
        } else {
            long long f = e - nK - nF - nE;
            int row = (int)(f / (4 * no)), col = (int)(f % (4 * no));
            int rho = row / no, o = row % no, i = col / no, o2 = col % no;
            double2 ax = pml_alpha_f(cd.own_lo + o2 - p + 1.0, cd.w, p, h, Cp, omega);
            double2 gam = cdiv(make_double2(-1.0, 0.0), h2 * ax);
            double2 g = Xat(row_node(cd, rho, p), cd.own_lo + o, 4 * nz + k_src(i) * no + o2);
            S[cd.S_off + f] = k_sgn(i) * (g * gam);
        }
    }
}

// Diagonal block of interface j: A_j = I - [K_j(w-rows, x_j part); K_{j+1}(1-rows, x_j part)]
__global__ void k_inner_diag(const LayerDesc *__restrict__ layers, const CellDesc *__restrict__ cells,
                             const double2 *__restrict__ K, double2 *W, int j) {
    const LayerDesc &ld = layers[blockIdx.y];
    if (j >= ld.C - 1) return;
    const int nz = ld.nz, n2 = 2 * nz;
    const CellDesc &ca = cells[ld.cell0 + j], &cb = cells[ld.cell0 + j + 1];
    double2 *A = W + ld.W_off + (long long)j * n2 * n2;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n2 * n2; e += gridDim.x * blockDim.x) {
        int m = e / n2, k = e % n2;
        double2 v = (m < nz) ? K[ca.K_off + (long long)(nz + m) * 4 * nz + 2 * nz + k]
                             : K[cb.K_off + (long long)(m - nz) * 4 * nz + k];
        double2 d = make_double2(m == k ? 1.0 : 0.0, 0.0);
        A[e] = d - v;
    }
}

// Z_j = K_j(w-rows, x_{j-1} part)  (nz x 2nz), stored in slot j of a buffer laid out like P
__global__ void k_inner_z(const LayerDesc *__restrict__ layers, const CellDesc *__restrict__ cells,
                          const double2 *__restrict__ K, double2 *Z, int j) {
    const LayerDesc &ld = layers[blockIdx.y];
    if (j >= ld.C - 1 || j == 0) return;
    const int nz = ld.nz, n2 = 2 * nz;
    const CellDesc &ca = cells[ld.cell0 + j];
    double2 *Zj = Z + ld.P_off + (long long)j * n2 * n2;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nz * n2; e += gridDim.x * blockDim.x) {
        int m = e / n2, k = e % n2;
        Zj[e] = K[ca.K_off + (long long)(nz + m) * 4 * nz + k];
    }
}

__global__ void k_d2f(const double2 *__restrict__ a, float2 *b, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

static void to_f32(const double2 *a, float2 *b, long long n, cudaStream_t st, int *nl) {
    if (n <= 0) return;
    k_d2f<<<1024, 256, 0, st>>>(a, b, n);
    HZ_CU(cudaGetLastError());
    (*nl)++;
}

static void check_info(hz_ctx *c, int *d_info, cudaStream_t st, const char *what) {
    int info = 0;
    HZ_CU(cudaMemcpyAsync(&info, d_info, sizeof(int), cudaMemcpyDeviceToHost, st));
    HZ_CU(cudaStreamSynchronize(st));
    if (c->fault == hz_ctx::FAULT_SINGULAR && !info) info = -1;  // as if a pivot had been exactly zero
    if (info) {
        char b[200];
        snprintf(b, sizeof b, "%s: zero pivot (code %d)", what, info);
        throw HzError(HZ_ESINGULAR, b);
    }
}

template <class T2> static T2 *alloc_n(hz_ctx *c, long long n) { return (T2 *)c->dalloc(sizeof(T2) * std::max(n, 1LL)); }

// ------------------------------------------- compressed-block LU (offline) ---
// Low-rank form of the inner block-LU factors P_j and V_j (Section 4.2.2, with
// the compression of Section 4.3): each is the cell's Green's function between
// its two sides, of low numerical rank.  For every block A (n2 x n2) an
// adaptive randomized range finder (Halko, Martinsson & Tropp 2011, Alg. 4.2)
// builds an orthonormal Q with ||A - Q Q^H A||_F <= eps ||A||_F: samples
// y = A w of complex Gaussian vectors w are orthogonalised against the columns
// found so far (classical Gram-Schmidt, two passes); a sample whose remainder
// is above the threshold adds a column, and four consecutive ones below it end
// the search.  Then B = Q^H A, and the bound is checked explicitly.

// complex Gaussian entries (real and imaginary parts N(0, 1/2)) from a counter-based
// generator (SplitMix64 of the entry index, Box-Muller)
__device__ inline unsigned long long smix(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__global__ void k_gauss(double2 *w, long long n, unsigned long long seed) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long a = smix(seed + 2 * (unsigned long long)i), b = smix(seed + 2 * (unsigned long long)i + 1);
        const double u1 = ((a >> 11) + 1.0) * (1.0 / 9007199254740993.0), u2 = (b >> 11) * (1.0 / 9007199254740992.0);
        const double r = sqrt(-log(u1)), t = 6.283185307179586 * u2;
        w[i] = make_double2(r * cos(t), r * sin(t));
    }
}

// sum of |a|^2 over the n2 x n2 block at mats[b] (one block per CTA)
__global__ void k_fro2(double2 *const *mats, const int *n2s, double *out) {
    const double2 *A = mats[blockIdx.x];
    const long long n = (long long)n2s[blockIdx.x] * n2s[blockIdx.x];
    double s = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) s += A[i].x * A[i].x + A[i].y * A[i].y;
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

// sum of |a - d|^2 of two n2 x n2 blocks (one pair per CTA)
__global__ void k_diff2(double2 *const *mats, double2 *const *dmats, const int *n2s, double *out) {
    const double2 *A = mats[blockIdx.x], *D = dmats[blockIdx.x];
    const long long n = (long long)n2s[blockIdx.x] * n2s[blockIdx.x];
    double s = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        const double x = A[i].x - D[i].x, y = A[i].y - D[i].y;
        s += x * x + y * y;
    }
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

// range finder of one block per CTA on its samples Y ([n2][kmax], y_c = A w_c in
// column c): the accepted columns, orthonormal, are compacted to the left of Y and
// the rest zeroed; kout = their number, or -1 if kmax samples did not capture the
// range.  thr = threshold on a sample's remainder.
__global__ void __launch_bounds__(256) k_range(double2 *const *Ys, const int *n2s, int kmax, int vlen,
                                               const double *thr, int *kout) {
    extern __shared__ double2 rsm[];
    double2 *v = rsm;         // [vlen >= n2]
    double2 *d = rsm + vlen;  // [kmax]
    __shared__ double red[8];
    __shared__ int s_acc;
    double2 *Y = Ys[blockIdx.x];
    const int n2 = n2s[blockIdx.x];
    const double th = thr[blockIdx.x];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int k = 0, small = 0;
    for (int c = 0; c < kmax && small < 4; c++) {
        for (int r = tid; r < n2; r += 256) v[r] = Y[(long long)r * kmax + c];
        __syncthreads();
        for (int pass = 0; pass < 2; pass++) {
            for (int i = warp; i < k; i += 8) {  // d_i = q_i^H v
                double2 a = make_double2(0.0, 0.0);
                for (int r = lane; r < n2; r += 32) {
                    const double2 q = Y[(long long)r * kmax + i], x = v[r];
                    a.x += q.x * x.x + q.y * x.y;
                    a.y += q.x * x.y - q.y * x.x;
                }
                for (int o = 16; o > 0; o >>= 1) {
                    a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
                    a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
                }
                if (lane == 0) d[i] = a;
            }
            __syncthreads();
            for (int r = tid; r < n2; r += 256) {  // v -= Q d
                double2 a = v[r];
                for (int i = 0; i < k; i++) {
                    const double2 q = Y[(long long)r * kmax + i], di = d[i];
                    a.x -= q.x * di.x - q.y * di.y;
                    a.y -= q.x * di.y + q.y * di.x;
                }
                v[r] = a;
            }
            __syncthreads();
        }
        double s = 0.0;
        for (int r = tid; r < n2; r += 256) s += v[r].x * v[r].x + v[r].y * v[r].y;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[warp] = s;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < 8; w++) t += red[w];
            s_acc = sqrt(t) > th ? 1 : 0;
            red[0] = sqrt(t);
        }
        __syncthreads();
        if (s_acc) {
            const double inv = 1.0 / red[0];
            for (int r = tid; r < n2; r += 256) Y[(long long)r * kmax + k] = make_double2(v[r].x * inv, v[r].y * inv);
            k++;
            small = 0;
        } else {
            small++;
        }
        __syncthreads();
    }
    for (int e = tid; e < n2 * (kmax - k); e += 256) {
        const int r = e / (kmax - k), cc = k + e % (kmax - k);
        Y[(long long)r * kmax + cc] = make_double2(0.0, 0.0);
    }
    if (tid == 0) kout[blockIdx.x] = small >= 4 ? k : -1;
}

// QH = Q^H (kmax x n2) of Q ([n2][kmax])
__global__ void k_conj_t(double2 *const *Qs, double2 *const *QHs, const int *n2s, int kmax) {
    const double2 *Q = Qs[blockIdx.y];
    double2 *QH = QHs[blockIdx.y];
    const int n2 = n2s[blockIdx.y];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n2 * kmax; e += gridDim.x * blockDim.x) {
        const int i = e / n2, r = e % n2;
        const double2 q = Q[(long long)r * kmax + i];
        QH[e] = make_double2(q.x, -q.y);
    }
}

// UX_j = [QP_j QV_j] (n2 x 2r): columns 0..r-1 from QP_j, r..2r-1 from QV_j (null: zero)
__global__ void k_build_ux(double2 *const *qp, double2 *const *qv, double2 *const *ux, const int *n2s, int kmax, int r) {
    const double2 *P = qp[blockIdx.y], *V = qv[blockIdx.y];
    double2 *U = ux[blockIdx.y];
    const int n2 = n2s[blockIdx.y];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n2 * 2 * r; e += gridDim.x * blockDim.x) {
        const int row = e / (2 * r), cc = e % (2 * r);
        const double2 *src = cc < r ? P : V;
        const int col = cc < r ? cc : cc - r;
        U[e] = src ? src[(long long)row * kmax + col] : make_double2(0.0, 0.0);
    }
}

// blocks of the recursion matrices stored transposed (column i of a block contiguous),
// so that the threads of a warp, which take consecutive rows, read consecutive words:
// block b is rows[b] x cols[b] at off[b] of src, written cols[b] x rows[b] at off[b] of dst
__global__ void k_block_t(const double2 *__restrict__ src, double2 *dst, const long long *off, const int *rows,
                          const int *cols) {
    const long long o = off[blockIdx.y];
    const int R = rows[blockIdx.y], Cn = cols[blockIdx.y];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < R * Cn; e += gridDim.x * blockDim.x) {
        const int i = e / Cn, k = e % Cn;
        dst[o + (long long)k * R + i] = src[o + e];
    }
}

// run a host-built list of FP64 products (64 x 32 tiles, no split)
// Unit columns that start the recursion on the identity (one thread per unit):
// for layer q, lam[q] (rows [J][2r], Nc = 2rJ columns) gets t_{j+1} row i <- column
// 2rj + i (j = 0..J-2), and u[q] ([J][r] rows) gets u_j row i <- column 2rj + r + i
__global__ void k_lam_init(double2 *const *lam, double2 *const *u, int r, int J) {
    const int q = blockIdx.y, Nc = 2 * r * J;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < J * r; e += gridDim.x * blockDim.x) {
        const int j = e / r, i = e % r;
        if (j <= J - 2) lam[q][((long long)(j + 1) * 2 * r + i) * Nc + (long long)j * 2 * r + i] = make_double2(1.0, 0.0);
        u[q][((long long)j * r + i) * Nc + (long long)j * 2 * r + r + i] = make_double2(1.0, 0.0);
    }
}

static void run_list64(hz_ctx *c, const std::vector<GemmProb<double2>> &v) {
    if (v.empty()) return;
    int mt = 0;
    for (const auto &g : v) mt = std::max(mt, gemm_tiles(g.M, g.N, 0));
    GemmProb<double2> *d = (GemmProb<double2> *)c->dalloc(sizeof(GemmProb<double2>) * v.size());
    HZ_CU(cudaMemcpyAsync(d, v.data(), sizeof(GemmProb<double2>) * v.size(), cudaMemcpyHostToDevice, c->st));
    launch_gemm<double2>(d, (int)v.size(), mt, 1, nullptr, nullptr, c->st, &c->nl);
    HZ_CU(cudaStreamSynchronize(c->st));
    c->dfree(d);
}
static GemmProb<double2> prob64(const double2 *A, long long lda, int M, int K, int N, const double2 *X, long long ldx,
                                double2 *Y, long long ldy) {
    GemmProb<double2> g{};
    g.A = A;
    g.lda = lda;
    g.M = M;
    g.K = K;
    g.N = N;
    g.xseg = g.yseg = 1 << 30;
    g.X[0] = X;
    g.ldx = ldx;
    g.Y[0] = Y;
    g.ldy = ldy;
    g.beta = 0;
    g.alpha = 1.f;
    return g;
}

// Compress the P / V factors of layers `lsub` (FP64, full-size arrays Pm / Vi / Wi)
// and write the compressed operators STW / UX / MRN (FP64, full-size arrays).  The
// first call fixes the rank r of the context (largest block rank, rounded up to a
// multiple of 8) and the layers' offsets; later calls (local updates) must fit in it.
static void compress_inner(hz_ctx *c, const std::vector<int> &lays, std::vector<LayerDesc> &lsub, const double2 *Wi,
                           const double2 *Pm, const double2 *Vi, double2 *&STW, double2 *&UX, double2 *&MRN,
                           double2 *&LAM, bool first) {
    const double eps = c->opts.compress;
    const int C = c->C, J = C - 1;
    if (J < 2) return;
    int max_n2 = 0;
    for (const LayerDesc &ld : lsub) max_n2 = std::max(max_n2, 2 * ld.nz);
    const int kmax = std::min(max_n2, 128);
    // the blocks: P_j (j = 1..J-1) and V_j (j = 0..J-2) of every layer
    struct Blk {
        int q, j, isV;
    };
    std::vector<Blk> blks;
    for (int q = 0; q < (int)lsub.size(); q++)
        for (int j = 0; j < J; j++) {
            if (j >= 1) blks.push_back({q, j, 0});
            if (j <= J - 2) blks.push_back({q, j, 1});
        }
    const int nb = (int)blks.size();
    std::vector<double2 *> A(nb), Y(nb), QH(nb), Bm(nb), D(nb);
    std::vector<int> n2s(nb);
    double2 *Om = alloc_n<double2>(c, (long long)max_n2 * kmax);
    k_gauss<<<256, 256, 0, c->st>>>(Om, (long long)max_n2 * kmax, 0x5eedull);
    HZ_CU(cudaGetLastError());
    c->nl++;
    long long per = 0;  // scratch per block: Y, QH, Bm, D
    per = (long long)max_n2 * kmax * 3 + (long long)max_n2 * max_n2;
    double2 *scr = alloc_n<double2>(c, per * nb);
    HZ_CU(cudaMemsetAsync(scr, 0, sizeof(double2) * per * nb, c->st));
    for (int b = 0; b < nb; b++) {
        const LayerDesc &ld = lsub[blks[b].q];
        const int n2 = 2 * ld.nz;
        n2s[b] = n2;
        A[b] = const_cast<double2 *>((blks[b].isV ? Vi + ld.V_off : Pm + ld.P_off) + (long long)blks[b].j * n2 * n2);
        Y[b] = scr + per * b;
        QH[b] = Y[b] + (long long)max_n2 * kmax;
        Bm[b] = QH[b] + (long long)max_n2 * kmax;
        D[b] = Bm[b] + (long long)max_n2 * kmax;
    }
    double2 **dA = (double2 **)c->dalloc(sizeof(double2 *) * nb * 3);
    double2 **dY = dA + nb, **dQH = dA + 2 * nb;
    int *dn = (int *)c->dalloc(sizeof(int) * nb * 2);
    int *dk = dn + nb;
    double *dv = (double *)c->dalloc(sizeof(double) * nb * 2);
    HZ_CU(cudaMemcpyAsync(dA, A.data(), sizeof(double2 *) * nb, cudaMemcpyHostToDevice, c->st));
    HZ_CU(cudaMemcpyAsync(dY, Y.data(), sizeof(double2 *) * nb, cudaMemcpyHostToDevice, c->st));
    HZ_CU(cudaMemcpyAsync(dQH, QH.data(), sizeof(double2 *) * nb, cudaMemcpyHostToDevice, c->st));
    HZ_CU(cudaMemcpyAsync(dn, n2s.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, c->st));
    k_fro2<<<nb, 256, 0, c->st>>>(dA, dn, dv);
    HZ_CU(cudaGetLastError());
    c->nl++;
    std::vector<double> nrm2(nb), thr(nb);
    HZ_CU(cudaMemcpyAsync(nrm2.data(), dv, sizeof(double) * nb, cudaMemcpyDeviceToHost, c->st));
    HZ_CU(cudaStreamSynchronize(c->st));
    // a sample's remainder estimates ||(I - Q Q^H) A||_F; stop well below the target
    for (int b = 0; b < nb; b++) thr[b] = 0.25 * eps * std::sqrt(nrm2[b]);
    HZ_CU(cudaMemcpyAsync(dv + nb, thr.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, c->st));
    {  // samples Y = A W
        std::vector<GemmProb<double2>> v;
        for (int b = 0; b < nb; b++) v.push_back(prob64(A[b], n2s[b], n2s[b], n2s[b], kmax, Om, kmax, Y[b], kmax));
        run_list64(c, v);
    }
    const size_t rsm = sizeof(double2) * (max_n2 + kmax);
    if (rsm > 48 * 1024) HZ_CU(cudaFuncSetAttribute(k_range, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm));
    k_range<<<nb, 256, rsm, c->st>>>(dY, dn, kmax, max_n2, dv + nb, dk);
    HZ_CU(cudaGetLastError());
    c->nl++;
    std::vector<int> ks(nb);
    HZ_CU(cudaMemcpyAsync(ks.data(), dk, sizeof(int) * nb, cudaMemcpyDeviceToHost, c->st));
    HZ_CU(cudaStreamSynchronize(c->st));
    int kbig = 0;
    for (int b = 0; b < nb; b++) {
        if (ks[b] < 0)
            throw HzError(HZ_EINVAL, "compressed-block LU: a factor's numerical rank exceeds " + std::to_string(kmax) +
                                         " at this tolerance; use a larger tolerance or dense factors");
        kbig = std::max(kbig, ks[b]);
    }
    k_conj_t<<<dim3(64, nb), 256, 0, c->st>>>(dY, dQH, dn, kmax);
    HZ_CU(cudaGetLastError());
    c->nl++;
    {  // B = Q^H A, then D = Q B for the explicit check
        std::vector<GemmProb<double2>> v;
        for (int b = 0; b < nb; b++) v.push_back(prob64(QH[b], n2s[b], kmax, n2s[b], n2s[b], A[b], n2s[b], Bm[b], n2s[b]));
        run_list64(c, v);
        v.clear();
        for (int b = 0; b < nb; b++) v.push_back(prob64(Y[b], kmax, n2s[b], kmax, n2s[b], Bm[b], n2s[b], D[b], n2s[b]));
        run_list64(c, v);
    }
    double2 **dD = dQH;  // reuse the pointer table
    HZ_CU(cudaMemcpyAsync(dD, D.data(), sizeof(double2 *) * nb, cudaMemcpyHostToDevice, c->st));
    k_diff2<<<nb, 256, 0, c->st>>>(dA, dD, dn, dv);
    HZ_CU(cudaGetLastError());
    c->nl++;
    std::vector<double> err2(nb);
    HZ_CU(cudaMemcpyAsync(err2.data(), dv, sizeof(double) * nb, cudaMemcpyDeviceToHost, c->st));
    HZ_CU(cudaStreamSynchronize(c->st));
    for (int b = 0; b < nb; b++)
        if (!(err2[b] <= eps * eps * nrm2[b]))
            throw HzError(HZ_EINVAL, "compressed-block LU: the low-rank form of a factor missed its tolerance");
    // the rank and layout (fixed by the first factorization)
    if (first) {
        c->lr_r = std::min(kmax, std::max(8, (kbig + 7) / 8 * 8));
        const int r = c->lr_r;
        long long lo = 0, mo = 0, ao = 0, la = 0;
        for (LayerDesc &ld : c->layers) {
            ld.lr_off = lo;
            lo += (long long)J * 2 * r * 2 * ld.nz;
            ld.m_off = mo;
            mo += (long long)J * 3 * r * r;
            ld.ac_off = ao;
            ao += (long long)J * 2 * r;
            ld.lam_off = la;
            la += (long long)(2 * r * J) * (2 * r * J);
        }
        c->tot_lr = lo;
        c->tot_m = mo;
        c->tot_ac = ao;
        c->tot_lam = la;
        HZ_CU(cudaMemcpyAsync(c->d_layers, c->layers.data(), sizeof(LayerDesc) * c->layers.size(),
                              cudaMemcpyHostToDevice, c->st));
        for (int q = 0; q < (int)lsub.size(); q++) lsub[q] = c->layers[lays[q]];
    } else if (kbig > c->lr_r) {
        throw HzError(HZ_EINVAL, "compressed-block LU: the updated medium needs a larger rank than the first "
                                 "factorization; factor afresh");
    }
    const int r = c->lr_r;
    if (r > kmax) throw HzError(HZ_EINVAL, "compressed-block LU: rank layout larger than the samples");
    // FP64 operator arrays (full size; null: allocated here)
    if (!STW) STW = alloc_n<double2>(c, c->tot_lr);
    if (!UX) UX = alloc_n<double2>(c, c->tot_lr);
    if (!MRN) MRN = alloc_n<double2>(c, c->tot_m);
    if (!LAM) LAM = alloc_n<double2>(c, c->tot_lam);
    // STW_j = [BP_{j+1} W_j; BV_{j-1} W_j], UX_j = [QP_j QV_j], and the r x r matrices of the
    // recursion in the order of its steps: forward step j (1..J-1) at (j-1) 2r^2 holds
    // [M_{j+1}; R_{j-1}] (M_j = BP_j QP_{j-1}, R_j = BV_j QP_{j+1}; M_J = 0), backward step j
    // (J-2..1) at (J-1) 2r^2 + (J-2-j) r^2 holds N_{j-1} (N_j = BV_j QV_{j+1}); each step's
    // block is stored transposed
    auto blk = [&](int q, int j, int isV) {
        for (int b = 0; b < nb; b++)
            if (blks[b].q == q && blks[b].j == j && blks[b].isV == isV) return b;
        return -1;
    };
    for (const LayerDesc &ld : lsub) {
        HZ_CU(cudaMemsetAsync(STW + ld.lr_off, 0, sizeof(double2) * (long long)J * 2 * r * 2 * ld.nz, c->st));
        HZ_CU(cudaMemsetAsync(MRN + ld.m_off, 0, sizeof(double2) * (long long)J * 3 * r * r, c->st));
    }
    std::vector<GemmProb<double2>> v;
    std::vector<double2 *> qp, qv, ux;
    std::vector<int> uxn;
    for (int q = 0; q < (int)lsub.size(); q++) {
        const LayerDesc &ld = lsub[q];
        const int n2 = 2 * ld.nz;
        for (int j = 0; j < J; j++) {
            const double2 *Wj = Wi + ld.W_off + (long long)j * n2 * n2;
            double2 *stw = STW + ld.lr_off + (long long)j * 2 * r * n2;
            double2 *mrn = MRN + ld.m_off + (long long)j * 3 * r * r;
            const int bp1 = j + 1 <= J - 1 ? blk(q, j + 1, 0) : -1, bvm1 = j >= 1 ? blk(q, j - 1, 1) : -1;
            if (bp1 >= 0) v.push_back(prob64(Bm[bp1], n2, r, n2, n2, Wj, n2, stw, n2));
            if (bvm1 >= 0) v.push_back(prob64(Bm[bvm1], n2, r, n2, n2, Wj, n2, stw + (long long)r * n2, n2));
            const int bp = j >= 1 ? blk(q, j, 0) : -1, bv = j <= J - 2 ? blk(q, j, 1) : -1;
            const int bpm = j >= 2 ? blk(q, j - 1, 0) : -1;
            const int bpp = j + 1 <= J - 1 ? blk(q, j + 1, 0) : -1, bvp = j + 1 <= J - 2 ? blk(q, j + 1, 1) : -1;
            const double2 *m0 = MRN + ld.m_off;
            const long long rr = (long long)r * r;
            if (bp >= 0 && bpm >= 0)  // M_j -> forward step j-1
                v.push_back(prob64(Bm[bp], n2, r, n2, r, Y[bpm], kmax, const_cast<double2 *>(m0) + (j - 2) * 2 * rr, r));
            if (bv >= 0 && bpp >= 0)  // R_j -> forward step j+1
                v.push_back(prob64(Bm[bv], n2, r, n2, r, Y[bpp], kmax, const_cast<double2 *>(m0) + j * 2 * rr + rr, r));
            if (bv >= 0 && bvp >= 0)  // N_j -> backward step j+1
                v.push_back(prob64(Bm[bv], n2, r, n2, r, Y[bvp], kmax,
                                   const_cast<double2 *>(m0) + (long long)(J - 1) * 2 * rr + (J - 3 - j) * rr, r));
            (void)mrn;
            qp.push_back(bp >= 0 ? Y[bp] : nullptr);
            qv.push_back(bv >= 0 ? Y[bv] : nullptr);
            ux.push_back(UX + ld.lr_off + (long long)j * n2 * 2 * r);
            uxn.push_back(n2);
        }
    }
    run_list64(c, v);
    {  // LAM: the recursion below run on the identity (all 2rJ unit columns at once), as
       // FP64 products over the layers, one list per step, with the step matrices still
       // stored row-major
        const int Nc = 2 * r * J, nq = (int)lsub.size();
        const long long rr = (long long)r * r, unit = (long long)r * Nc;
        double2 *U = alloc_n<double2>(c, (long long)nq * J * unit);
        HZ_CU(cudaMemsetAsync(U, 0, sizeof(double2) * nq * J * unit, c->st));
        std::vector<double2 *> lp(nq), up(nq);
        for (int q = 0; q < nq; q++) {
            lp[q] = LAM + lsub[q].lam_off;
            up[q] = U + (long long)q * J * unit;
            HZ_CU(cudaMemsetAsync(lp[q], 0, sizeof(double2) * Nc * Nc, c->st));
        }
        double2 **dp = (double2 **)c->dalloc(sizeof(double2 *) * 2 * nq);
        HZ_CU(cudaMemcpyAsync(dp, lp.data(), sizeof(double2 *) * nq, cudaMemcpyHostToDevice, c->st));
        HZ_CU(cudaMemcpyAsync(dp + nq, up.data(), sizeof(double2 *) * nq, cudaMemcpyHostToDevice, c->st));
        k_lam_init<<<dim3(8, nq), 256, 0, c->st>>>(dp, dp + nq, r, J);
        HZ_CU(cudaGetLastError());
        c->nl++;
        // forward: [t_{j+1}; u_j] += [M_{j+1}; R_{j-1}] t_j (t_J is not kept)
        for (int j = 1; j <= J - 1; j++) {
            std::vector<GemmProb<double2>> w;
            for (int q = 0; q < nq; q++) {
                const double2 *blk = MRN + lsub[q].m_off + (long long)(j - 1) * 2 * rr;
                const double2 *tj = lp[q] + (long long)j * 2 * r * Nc;
                if (j + 1 <= J - 1) {
                    GemmProb<double2> g = prob64(blk, r, 2 * r, r, Nc, tj, Nc, lp[q] + (long long)(j + 1) * 2 * r * Nc, Nc);
                    g.yseg = r;
                    g.Y[1] = up[q] + (long long)j * unit;
                    g.beta = 1;
                    w.push_back(g);
                } else {
                    GemmProb<double2> g = prob64(blk + rr, r, r, r, Nc, tj, Nc, up[q] + (long long)j * unit, Nc);
                    g.beta = 1;
                    w.push_back(g);
                }
            }
            run_list64(c, w);
        }
        // backward: s_{j-1} = u_j + N_{j-1} s_j, from s_{J-2} = u_{J-1} (s_{J-1} = 0)
        for (int q = 0; q < nq; q++)
            HZ_CU(cudaMemcpy2DAsync(lp[q] + (long long)r * Nc, sizeof(double2) * 2 * unit, up[q] + unit,
                                    sizeof(double2) * unit, sizeof(double2) * unit, J - 1, cudaMemcpyDeviceToDevice,
                                    c->st));
        for (int j = J - 2; j >= 1; j--) {
            std::vector<GemmProb<double2>> w;
            for (int q = 0; q < nq; q++) {
                const double2 *nb = MRN + lsub[q].m_off + (long long)(J - 1) * 2 * rr + (long long)(J - 2 - j) * rr;
                GemmProb<double2> g = prob64(nb, r, r, r, Nc, lp[q] + ((long long)j * 2 * r + r) * Nc, Nc,
                                             lp[q] + ((long long)(j - 1) * 2 * r + r) * Nc, Nc);
                g.beta = 1;
                w.push_back(g);
            }
            run_list64(c, w);
        }
        HZ_CU(cudaStreamSynchronize(c->st));
        c->dfree(dp);
        c->dfree(U);
    }
    {  // each step's matrix transposed in place (through a copy of the layers' ranges)
        std::vector<long long> offs;
        std::vector<int> rws, cls;
        long long tot = 0;
        for (const LayerDesc &ld : lsub) {
            const long long rr = (long long)r * r, base = ld.m_off;
            for (int j = 1; j <= J - 1; j++) {  // forward steps: [M; R], 2r x r
                offs.push_back(base + (long long)(j - 1) * 2 * rr);
                rws.push_back(2 * r);
                cls.push_back(r);
            }
            for (int b = 0; b < J - 2; b++) {  // backward steps: N, r x r
                offs.push_back(base + (long long)(J - 1) * 2 * rr + b * rr);
                rws.push_back(r);
                cls.push_back(r);
            }
            tot = std::max(tot, base + (long long)J * 3 * rr);
        }
        const int nbk = (int)offs.size();
        if (nbk > 0) {
            double2 *cp = alloc_n<double2>(c, tot);
            HZ_CU(cudaMemcpyAsync(cp, MRN, sizeof(double2) * tot, cudaMemcpyDeviceToDevice, c->st));
            long long *doff = (long long *)c->dalloc(sizeof(long long) * nbk);
            int *drc = (int *)c->dalloc(sizeof(int) * 2 * nbk);
            HZ_CU(cudaMemcpyAsync(doff, offs.data(), sizeof(long long) * nbk, cudaMemcpyHostToDevice, c->st));
            HZ_CU(cudaMemcpyAsync(drc, rws.data(), sizeof(int) * nbk, cudaMemcpyHostToDevice, c->st));
            HZ_CU(cudaMemcpyAsync(drc + nbk, cls.data(), sizeof(int) * nbk, cudaMemcpyHostToDevice, c->st));
            k_block_t<<<dim3(16, nbk), 256, 0, c->st>>>(cp, MRN, doff, drc, drc + nbk);
            HZ_CU(cudaGetLastError());
            c->nl++;
            HZ_CU(cudaStreamSynchronize(c->st));
            c->dfree(cp);
            c->dfree(doff);
            c->dfree(drc);
        }
    }
    const int nu = (int)ux.size();
    double2 **du = (double2 **)c->dalloc(sizeof(double2 *) * nu * 3);
    int *dun = (int *)c->dalloc(sizeof(int) * nu);
    HZ_CU(cudaMemcpyAsync(du, qp.data(), sizeof(double2 *) * nu, cudaMemcpyHostToDevice, c->st));
    HZ_CU(cudaMemcpyAsync(du + nu, qv.data(), sizeof(double2 *) * nu, cudaMemcpyHostToDevice, c->st));
    HZ_CU(cudaMemcpyAsync(du + 2 * nu, ux.data(), sizeof(double2 *) * nu, cudaMemcpyHostToDevice, c->st));
    HZ_CU(cudaMemcpyAsync(dun, uxn.data(), sizeof(int) * nu, cudaMemcpyHostToDevice, c->st));
    k_build_ux<<<dim3(32, nu), 256, 0, c->st>>>(du, du + nu, du + 2 * nu, dun, kmax, r);
    HZ_CU(cudaGetLastError());
    c->nl++;
    HZ_CU(cudaStreamSynchronize(c->st));
    for (void *q : {(void *)Om, (void *)scr, (void *)dA, (void *)dn, (void *)dv, (void *)du, (void *)dun}) c->dfree(q);
}


// P2 += S of each listed cell: S (4 no x 4 no, columns [q][no]) into the cell's own
// columns of its composite (columns [q][Lt], own columns at cl)
__global__ void k_add_s(const CellDesc *__restrict__ cells, const double2 *__restrict__ S, double2 *P2) {
    const CellDesc cd = cells[blockIdx.y];
    const int no = cd.no, w = 4 * no;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < w * w; e += gridDim.x * blockDim.x) {
        const int row = e / w, col = e % w, q = col / no, i = col % no;
        double2 &d = P2[cd.P2_off + (long long)row * 4 * cd.Lt + (long long)q * cd.Lt + cd.cl + i];
        d = d + S[cd.S_off + e];
    }
}

// The sweep step of a layer with the compressed-block LU, out += E x + S in with
// x_j = W_j g_j + UX_j ts_j, g = F in and ts = LAM (STW g), regrouped as three
// products: [out += P2 in, ac = P1 in] -> ts = LAM ac -> out += P3 ts, with the
// per-cell composites P2 = E W F + S, P1 = STW F and P3 = E UX formed here in FP64
// (layout in CellDesc).  The first call fixes their offsets; later calls (local
// updates) rewrite the listed layers' blocks in place.
static void compose_sweep(hz_ctx *c, const std::vector<int> &lays, const double2 *F, const double2 *E,
                          const double2 *S, const double2 *Wi, const double2 *STW, const double2 *UX, double2 *&P2,
                          double2 *&P3, double2 *&P1, bool first) {
    const int C = c->C, J = C - 1, r = c->lr_r;
    if (r <= 0 || J < 1) return;
    if (first) {
        long long o2 = 0, o3 = 0, o1 = 0;
        for (const LayerDesc &ld : c->layers)
            for (int cc = 0; cc < C; cc++) {
                CellDesc &cd = c->cells[ld.cell0 + cc];
                const int nol = cc > 0 ? c->cells[ld.cell0 + cc - 1].no : 0;
                const int nor = cc < C - 1 ? c->cells[ld.cell0 + cc + 1].no : 0;
                if (cc > 0) {  // owned ranges of neighbouring cells are adjacent
                    const CellDesc &pv = c->cells[ld.cell0 + cc - 1];
                    if (pv.t + pv.own_lo + pv.no != cd.t + cd.own_lo)
                        throw HzError(HZ_EINVAL, "sweep composites: owned column ranges are not adjacent");
                }
                cd.cl = nol;
                cd.Lt = nol + cd.no + nor;
                cd.P2_off = o2;
                o2 += 4LL * cd.no * 4 * cd.Lt;
                cd.P3_off = o3;
                o3 += 4LL * cd.no * 4 * r;
                cd.P1_off = o1;
                if (cc < C - 1) o1 += 2LL * r * 4 * (cd.no + nor);
            }
        c->tot_cp2 = o2;
        c->tot_cp3 = o3;
        c->tot_cp1 = o1;
        HZ_CU(cudaMemcpyAsync(c->d_cells, c->cells.data(), sizeof(CellDesc) * c->cells.size(),
                              cudaMemcpyHostToDevice, c->st));
    }
    if (!P2) P2 = alloc_n<double2>(c, c->tot_cp2);
    if (!P3) P3 = alloc_n<double2>(c, c->tot_cp3);
    if (!P1) P1 = alloc_n<double2>(c, std::max(c->tot_cp1, 1LL));
    // the listed layers' cells, their WF_j temporaries and zeroed composite blocks
    std::vector<CellDesc> cl;
    std::vector<long long> wfo;  // per listed interface: offset of WF_j in the temporary
    long long wft = 0;
    for (int l : lays) {
        const LayerDesc &ld = c->layers[l];
        for (int cc = 0; cc < C; cc++) {
            const CellDesc &cd = c->cells[ld.cell0 + cc];
            cl.push_back(cd);
            HZ_CU(cudaMemsetAsync(P2 + cd.P2_off, 0, sizeof(double2) * 16LL * cd.no * cd.Lt, c->st));
            HZ_CU(cudaMemsetAsync(P3 + cd.P3_off, 0, sizeof(double2) * 16LL * cd.no * r, c->st));
            if (cc < C - 1) {
                const CellDesc &cn = c->cells[ld.cell0 + cc + 1];
                wfo.push_back(wft);
                wft += 2LL * ld.nz * 4 * (cd.no + cn.no);
            }
        }
    }
    double2 *WF = alloc_n<double2>(c, std::max(wft, 1LL));
    // WF_j = [W_j(:, 0:nz) F_j^(1) | W_j(:, nz:2nz) F_{j+1}^(0)] (2nz x 4 (no_j + no_{j+1}));
    // P1_j = the same with STW_j, columns regrouped [q][no_j + no_{j+1}]
    std::vector<GemmProb<double2>> v1, vl, vr;
    int iw = 0;
    for (int l : lays) {
        const LayerDesc &ld = c->layers[l];
        const int nz = ld.nz, n2 = 2 * nz;
        for (int j = 0; j < J; j++, iw++) {
            const CellDesc &ca = c->cells[ld.cell0 + j], &cb = c->cells[ld.cell0 + j + 1];
            const int L2 = ca.no + cb.no, lw = 4 * L2;
            double2 *wf = WF + wfo[iw];
            const double2 *Wj = Wi + ld.W_off + (long long)j * n2 * n2;
            const double2 *Fa = F + ca.F_off + (long long)nz * 4 * ca.no;  // F_j^(1): rows nz..2nz
            const double2 *Fb = F + cb.F_off;                              // F_{j+1}^(0)
            v1.push_back(prob64(Wj, n2, n2, nz, 4 * ca.no, Fa, 4LL * ca.no, wf, lw));
            v1.push_back(prob64(Wj + nz, n2, n2, nz, 4 * cb.no, Fb, 4LL * cb.no, wf + 4 * ca.no, lw));
            const double2 *Sj = STW + ld.lr_off + (long long)j * 2 * r * n2;
            double2 *p1 = P1 + ca.P1_off;
            for (int q = 0; q < 4; q++) {
                v1.push_back(prob64(Sj, n2, 2 * r, nz, ca.no, Fa + (long long)q * ca.no, 4LL * ca.no,
                                    p1 + (long long)q * L2, lw));
                v1.push_back(prob64(Sj + nz, n2, 2 * r, nz, cb.no, Fb + (long long)q * cb.no, 4LL * cb.no,
                                    p1 + (long long)q * L2 + ca.no, lw));
            }
        }
    }
    run_list64(c, v1);
    // P2_c = E_c(:, 0:2nz) WF_{c-1} + E_c(:, 2nz:4nz) WF_c (+ S_c below), columns regrouped;
    // P3_c = [E_c(:, 0:2nz) UX_{c-1} | E_c(:, 2nz:4nz) UX_c]
    iw = 0;
    for (int l : lays) {
        const LayerDesc &ld = c->layers[l];
        const int nz = ld.nz, n2 = 2 * nz;
        for (int cc = 0; cc < C; cc++) {
            const CellDesc &cd = c->cells[ld.cell0 + cc];
            const double2 *El = E + cd.E_off, *Er = El + n2;
            const long long ldp = 4LL * cd.Lt;
            double2 *p2 = P2 + cd.P2_off, *p3 = P3 + cd.P3_off;
            if (cc > 0) {  // interface cc-1: cells cc-1 (range offset 0) and cc (offset cl)
                const CellDesc &cp = c->cells[ld.cell0 + cc - 1];
                const double2 *wf = WF + wfo[iw + cc - 1];
                const long long lw = 4LL * (cp.no + cd.no);
                for (int q = 0; q < 4; q++) {
                    vl.push_back(prob64(El, 2LL * n2, 4 * cd.no, n2, cp.no, wf + (long long)q * cp.no, lw,
                                        p2 + (long long)q * cd.Lt, ldp));
                    vl.push_back(prob64(El, 2LL * n2, 4 * cd.no, n2, cd.no, wf + 4 * cp.no + (long long)q * cd.no, lw,
                                        p2 + (long long)q * cd.Lt + cd.cl, ldp));
                }
                vl.push_back(prob64(El, 2LL * n2, 4 * cd.no, n2, 2 * r,
                                    UX + ld.lr_off + (long long)(cc - 1) * n2 * 2 * r, 2 * r, p3, 4 * r));
            }
            if (cc < C - 1) {  // interface cc: cells cc (offset cl) and cc+1 (offset cl + no)
                const CellDesc &cn = c->cells[ld.cell0 + cc + 1];
                const double2 *wf = WF + wfo[iw + cc];
                const long long lw = 4LL * (cd.no + cn.no);
                for (int q = 0; q < 4; q++) {
                    vr.push_back(prob64(Er, 2LL * n2, 4 * cd.no, n2, cd.no, wf + (long long)q * cd.no, lw,
                                        p2 + (long long)q * cd.Lt + cd.cl, ldp));
                    vr.push_back(prob64(Er, 2LL * n2, 4 * cd.no, n2, cn.no, wf + 4 * cd.no + (long long)q * cn.no, lw,
                                        p2 + (long long)q * cd.Lt + cd.cl + cd.no, ldp));
                }
                vr.push_back(prob64(Er, 2LL * n2, 4 * cd.no, n2, 2 * r, UX + ld.lr_off + (long long)cc * n2 * 2 * r,
                                    2 * r, p3 + 2 * r, 4 * r));
            }
        }
        iw += J;
    }
    for (auto *w : {&vl, &vr})
        for (auto &g : *w) g.beta = 1;  // the two interfaces of a cell meet in its own columns
    run_list64(c, vl);
    run_list64(c, vr);
    CellDesc *dcl = (CellDesc *)c->dalloc(sizeof(CellDesc) * cl.size());
    HZ_CU(cudaMemcpyAsync(dcl, cl.data(), sizeof(CellDesc) * cl.size(), cudaMemcpyHostToDevice, c->st));
    k_add_s<<<dim3(32, (unsigned)cl.size()), 256, 0, c->st>>>(dcl, S, P2);
    HZ_CU(cudaGetLastError());
    c->nl++;
    HZ_CU(cudaStreamSynchronize(c->st));
    c->dfree(dcl);
    c->dfree(WF);
}

// ---------------------------------------------------------- factor ---
// Factorization of the layers in `lays` (all layers on the first call, from
// hz_factor; the layers whose cells read a changed medium on a local update,
// from hz_update_model).  Every stage below works on those layers' cells only
// and writes the operators in place at their global offsets, so a local update
// leaves the other layers' operators exactly as they were.
void factor_layers(hz_ctx *c, const std::vector<int> &lays, bool first) {
    cudaStream_t st = c->st;
    int *nl = &c->nl;
    const int p = c->p, C = c->C;
    const int nlay = (int)lays.size();
    if (nlay == 0) return;
    std::vector<CellDesc> sub;
    std::vector<LayerDesc> lsub;
    for (int l : lays) {
        lsub.push_back(c->layers[l]);
        for (int cc = 0; cc < C; cc++) sub.push_back(c->cells[c->layers[l].cell0 + cc]);
    }
    const int nsub = (int)sub.size();
    CellDesc *d_sub = (CellDesc *)c->dalloc(sizeof(CellDesc) * nsub);
    HZ_CU(cudaMemcpyAsync(d_sub, sub.data(), sizeof(CellDesc) * nsub, cudaMemcpyHostToDevice, st));
    LayerDesc *d_lsub = (LayerDesc *)c->dalloc(sizeof(LayerDesc) * nlay);
    HZ_CU(cudaMemcpyAsync(d_lsub, lsub.data(), sizeof(LayerDesc) * nlay, cudaMemcpyHostToDevice, st));
    int *d_info = (int *)c->dalloc(sizeof(int));
    HZ_CU(cudaMemsetAsync(d_info, 0, sizeof(int), st));
    const bool mixed = c->mixed();
    // FP64 operators: the context's own in FP64 mode, full-size temporaries in mixed mode
    auto fp64_buf = [&](double2 *&keep, long long n, bool zero) {
        if (!mixed && !first) return keep;
        double2 *q = alloc_n<double2>(c, n);
        if (zero) HZ_CU(cudaMemsetAsync(q, 0, sizeof(double2) * std::max(n, 1LL), st));
        if (!mixed) keep = q;
        return q;
    };

    // 1. cell operators (row-scaled form) and block-tridiagonal inverses
    double2 *diag = alloc_n<double2>(c, c->tot_vol), *cxv = alloc_n<double2>(c, c->tot_vol);
    double2 *czv = fp64_buf(c->o64.cz, c->tot_vol, false);
    launch_cell_coeffs(d_sub, nsub, c->d_m, c->NX, c->omega, c->h, c->pml_C, p, diag, cxv, czv, st, nl);
    double2 *cellW = fp64_buf(c->o64.cellW, c->tot_W, true);  // row padding stays zero
    launch_cell_factor(d_sub, nsub, diag, cxv, czv, cellW, c->max_nx, d_info, st, nl);
    check_info(c, d_info, st, "cell factorization");
    c->dfree(diag);
    c->dfree(cxv);

    // 2. Green's blocks from unit-source cell solves, in groups of cells
    double2 *K = alloc_n<double2>(c, c->tot_K);
    double2 *F = fp64_buf(c->o64.F, c->tot_F, false), *E = fp64_buf(c->o64.E, c->tot_E, false);
    double2 *S = fp64_buf(c->o64.S, c->tot_S, false);
    {
        const long long budget = 3LL << 30;  // bytes of solution buffer per group
        int i0 = 0;
        while (i0 < nsub) {
            int Bg = 0;
            long long pts = 0;
            int i1 = i0;
            while (i1 < nsub) {
                const CellDesc &cd = sub[i1];
                int nb = 4 * cd.nz + 4 * cd.no;
                int Bn = std::max(Bg, nb);
                long long ptsn = pts + (long long)cd.nx * cd.nz;
                if (i1 > i0 && ptsn * Bn * 16 > budget) break;
                Bg = Bn;
                pts = ptsn;
                i1++;
            }
            std::vector<CellDesc> grp(sub.begin() + i0, sub.begin() + i1);
            long long off = 0;
            for (auto &cd : grp) {
                cd.vol_off = off;
                off += (long long)cd.nx * cd.nz;
            }
            // W / cz offsets stay global
            CellDesc *d_grp = (CellDesc *)c->dalloc(sizeof(CellDesc) * grp.size());
            HZ_CU(cudaMemcpyAsync(d_grp, grp.data(), sizeof(CellDesc) * grp.size(), cudaMemcpyHostToDevice, st));
            double2 *X = alloc_n<double2>(c, pts * Bg);
            HZ_CU(cudaMemsetAsync(X, 0, sizeof(double2) * pts * Bg, st));
            k_unit_sources<<<dim3((Bg + 255) / 256, (unsigned)grp.size()), 256, 0, st>>>(d_grp, X, Bg, p);
            HZ_CU(cudaGetLastError());
            (*nl)++;
            launch_cell_chain<double2>(d_grp, (int)grp.size(), cellW, czv, X, Bg, c->max_nx, st, nl);
            k_extract<<<dim3(256, (unsigned)grp.size()), 256, 0, st>>>(d_grp, X, Bg, p, c->h, c->pml_C, c->omega, K,
                                                                       F, E, S);
            HZ_CU(cudaGetLastError());
            (*nl)++;
            HZ_CU(cudaStreamSynchronize(st));
            c->dfree(X);
            c->dfree(d_grp);
            i0 = i1;
        }
    }

    // 3. inner block LU per layer: S_j = A_j - [Z_j V_{j-1}; 0], W_j = S_j^{-1},
    //    V_j = W_j(:, nz:2nz) K_{j+1}(1-rows, x_{j+1} part)
    double2 *Wi = fp64_buf(c->o64.W, c->tot_Wi, false), *Zi = alloc_n<double2>(c, c->tot_P);
    double2 *Pm = fp64_buf(c->o64.P, c->tot_P, false), *Vi = fp64_buf(c->o64.V, c->tot_V, false);
    if (C > 1) {
        GemmProb<double2> *d_pr = (GemmProb<double2> *)c->dalloc(sizeof(GemmProb<double2>) * nlay);
        double2 **d_mats = (double2 **)c->dalloc(sizeof(double2 *) * nlay);
        int *d_ns = (int *)c->dalloc(sizeof(int) * nlay);
        std::vector<GemmProb<double2>> pr(nlay);
        std::vector<double2 *> mats(nlay);
        std::vector<int> ns(nlay);
        int maxn2 = 0;
        for (const LayerDesc &ld : lsub) maxn2 = std::max(maxn2, 2 * ld.nz);
        for (int j = 0; j < C - 1; j++) {
            k_inner_diag<<<dim3(64, nlay), 256, 0, st>>>(d_lsub, c->d_cells, K, Wi, j);
            HZ_CU(cudaGetLastError());
            (*nl)++;
            k_inner_z<<<dim3(64, nlay), 256, 0, st>>>(d_lsub, c->d_cells, K, Zi, j);
            HZ_CU(cudaGetLastError());
            (*nl)++;
            if (j > 0) {  // S_j(a-rows) -= Z_j V_{j-1}
                int mt = 0;
                for (int q = 0; q < nlay; q++) {
                    const LayerDesc &ld = lsub[q];
                    const int nz = ld.nz, n2 = 2 * nz;
                    GemmProb<double2> g{};
                    g.A = Zi + ld.P_off + (long long)j * n2 * n2;
                    g.lda = n2;
                    g.M = nz;
                    g.K = n2;
                    g.N = n2;
                    g.xseg = g.yseg = 1 << 30;
                    g.X[0] = Vi + ld.V_off + (long long)(j - 1) * n2 * n2;
                    g.ldx = n2;
                    g.Y[0] = Wi + ld.W_off + (long long)j * n2 * n2;
                    g.ldy = n2;
                    g.beta = 1;
                    g.alpha = -1.f;
                    pr[q] = g;
                    mt = std::max(mt, ((nz + 63) / 64) * ((n2 + 31) / 32));
                }
                HZ_CU(cudaMemcpyAsync(d_pr, pr.data(), sizeof(GemmProb<double2>) * nlay, cudaMemcpyHostToDevice, st));
                launch_gemm<double2>(d_pr, nlay, mt, 1, nullptr, nullptr, st, nl);
            }
            for (int q = 0; q < nlay; q++) {
                const LayerDesc &ld = lsub[q];
                const long long n2 = 2LL * ld.nz;
                mats[q] = Wi + ld.W_off + j * n2 * n2;
                ns[q] = (int)n2;
            }
            HZ_CU(cudaMemcpyAsync(d_mats, mats.data(), sizeof(double2 *) * nlay, cudaMemcpyHostToDevice, st));
            HZ_CU(cudaMemcpyAsync(d_ns, ns.data(), sizeof(int) * nlay, cudaMemcpyHostToDevice, st));
            launch_gj_inverse(d_mats, d_ns, nlay, maxn2, d_info, st, nl);
            if (j > 0) {  // P_j = W_j(:, 0:nz) Z_j: the forward sweep becomes y_j = W_j g_j + P_j y_{j-1}
                int mt = 0;
                for (int q = 0; q < nlay; q++) {
                    const LayerDesc &ld = lsub[q];
                    const int nz = ld.nz, n2 = 2 * nz;
                    GemmProb<double2> g{};
                    g.A = Wi + ld.W_off + (long long)j * n2 * n2;
                    g.lda = n2;
                    g.M = n2;
                    g.K = nz;
                    g.N = n2;
                    g.xseg = g.yseg = 1 << 30;
                    g.X[0] = Zi + ld.P_off + (long long)j * n2 * n2;
                    g.ldx = n2;
                    g.Y[0] = Pm + ld.P_off + (long long)j * n2 * n2;
                    g.ldy = n2;
                    g.beta = 0;
                    g.alpha = 1.f;
                    pr[q] = g;
                    mt = std::max(mt, ((n2 + 63) / 64) * ((n2 + 31) / 32));
                }
                HZ_CU(cudaStreamSynchronize(st));  // pr is reused below
                HZ_CU(cudaMemcpyAsync(d_pr, pr.data(), sizeof(GemmProb<double2>) * nlay, cudaMemcpyHostToDevice, st));
                launch_gemm<double2>(d_pr, nlay, mt, 1, nullptr, nullptr, st, nl);
                HZ_CU(cudaStreamSynchronize(st));
            }
            if (j < C - 2) {  // V_j = W_j(:, nz:) K_{j+1}(1-rows, right part)
                int mt = 0;
                for (int q = 0; q < nlay; q++) {
                    const LayerDesc &ld = lsub[q];
                    const int nz = ld.nz, n2 = 2 * nz;
                    const CellDesc &cb = c->cells[ld.cell0 + j + 1];
                    GemmProb<double2> g{};
                    g.A = Wi + ld.W_off + (long long)j * n2 * n2 + nz;
                    g.lda = n2;
                    g.M = n2;
                    g.K = nz;
                    g.N = n2;
                    g.xseg = g.yseg = 1 << 30;
                    g.X[0] = K + cb.K_off + 2 * nz;
                    g.ldx = 4 * nz;
                    g.Y[0] = Vi + ld.V_off + (long long)j * n2 * n2;
                    g.ldy = n2;
                    g.beta = 0;
                    g.alpha = 1.f;
                    pr[q] = g;
                    mt = std::max(mt, ((n2 + 63) / 64) * ((n2 + 31) / 32));
                }
                HZ_CU(cudaMemcpyAsync(d_pr, pr.data(), sizeof(GemmProb<double2>) * nlay, cudaMemcpyHostToDevice, st));
                launch_gemm<double2>(d_pr, nlay, mt, 1, nullptr, nullptr, st, nl);
            }
            HZ_CU(cudaStreamSynchronize(st));  // host vectors reused next step
        }
        check_info(c, d_info, st, "inner block LU");
        c->dfree(d_pr);
        c->dfree(d_mats);
        c->dfree(d_ns);
    }
    c->dfree(K);
    c->dfree(Zi);

    // 3b. compressed-block LU: low-rank P_j, V_j and the operators of the r-vector recursion
    double2 *STW64 = nullptr, *UX64 = nullptr, *MRN64 = nullptr, *LAM64 = nullptr;
    if (c->opts.compress > 0 && C > 2) {
        if (!mixed) {  // kept by the context in FP64 (allocated by the first call)
            STW64 = c->o64.STW;
            UX64 = c->o64.UX;
            MRN64 = c->o64.MRN;
            LAM64 = c->o64.LAM;
        }
        compress_inner(c, lays, lsub, Wi, Pm, Vi, STW64, UX64, MRN64, LAM64, first);
        if (!mixed) {
            c->o64.STW = STW64;
            c->o64.UX = UX64;
            c->o64.MRN = MRN64;
            c->o64.LAM = LAM64;
        }
    }
    // 3c. the sweep-step composites of the compressed-block LU
    double2 *CP2_64 = nullptr, *CP3_64 = nullptr, *CP1_64 = nullptr;
    if (c->lr_r > 0 && STW64) {
        if (!mixed) {
            CP2_64 = c->o64.CP2;
            CP3_64 = c->o64.CP3;
            CP1_64 = c->o64.CP1;
        }
        compose_sweep(c, lays, F, E, S, Wi, STW64, UX64, CP2_64, CP3_64, CP1_64, first);
        if (!mixed) {
            c->o64.CP2 = CP2_64;
            c->o64.CP3 = CP3_64;
            c->o64.CP1 = CP1_64;
        }
    }

    // 4. mixed precision: the working-precision copies of these layers' operators
    if (mixed) {
        auto &o = c->o32;
        if (first) {
            o.cellW = alloc_n<float2>(c, c->tot_W);
            o.cz = alloc_n<float2>(c, c->tot_vol);
            o.F = alloc_n<float2>(c, c->tot_F);
            o.E = alloc_n<float2>(c, c->tot_E);
            o.S = alloc_n<float2>(c, c->tot_S);
            o.W = alloc_n<float2>(c, c->tot_Wi);
            o.P = alloc_n<float2>(c, c->tot_P);
            o.V = alloc_n<float2>(c, c->tot_V);
            to_f32(cellW, o.cellW, c->tot_W, st, nl);
            to_f32(czv, o.cz, c->tot_vol, st, nl);
            to_f32(F, o.F, c->tot_F, st, nl);
            to_f32(E, o.E, c->tot_E, st, nl);
            to_f32(S, o.S, c->tot_S, st, nl);
            to_f32(Wi, o.W, c->tot_Wi, st, nl);
            to_f32(Pm, o.P, c->tot_P, st, nl);
            to_f32(Vi, o.V, c->tot_V, st, nl);
        } else {
            for (const CellDesc &cd : sub) {
                const long long nb = (long long)cd.nz * cd.nx * cd.ldw;
                to_f32(cellW + cd.w_off, o.cellW + cd.w_off, nb, st, nl);
                to_f32(czv + cd.cz_off, o.cz + cd.cz_off, (long long)cd.nx * cd.nz, st, nl);
                to_f32(F + cd.F_off, o.F + cd.F_off, 8LL * cd.nz * cd.no, st, nl);
                to_f32(E + cd.E_off, o.E + cd.E_off, 16LL * cd.no * cd.nz, st, nl);
                to_f32(S + cd.S_off, o.S + cd.S_off, 16LL * cd.no * cd.no, st, nl);
            }
            for (const LayerDesc &ld : lsub) {
                const long long n2 = 2LL * ld.nz, nb = (long long)std::max(C - 1, 0) * n2 * n2;
                to_f32(Wi + ld.W_off, o.W + ld.W_off, nb, st, nl);
                to_f32(Pm + ld.P_off, o.P + ld.P_off, nb, st, nl);
                to_f32(Vi + ld.V_off, o.V + ld.V_off, nb, st, nl);
            }
        }
        if (c->lr_r > 0 && STW64) {  // FP32 copies of the compressed-block LU operators
            const int J = C - 1, r = c->lr_r;
            if (first) {
                o.STW = alloc_n<float2>(c, c->tot_lr);
                o.UX = alloc_n<float2>(c, c->tot_lr);
                o.MRN = alloc_n<float2>(c, c->tot_m);
                o.LAM = alloc_n<float2>(c, c->tot_lam);
                to_f32(STW64, o.STW, c->tot_lr, st, nl);
                to_f32(UX64, o.UX, c->tot_lr, st, nl);
                to_f32(MRN64, o.MRN, c->tot_m, st, nl);
                to_f32(LAM64, o.LAM, c->tot_lam, st, nl);
                o.CP2 = alloc_n<float2>(c, c->tot_cp2);
                o.CP3 = alloc_n<float2>(c, c->tot_cp3);
                o.CP1 = alloc_n<float2>(c, std::max(c->tot_cp1, 1LL));
                to_f32(CP2_64, o.CP2, c->tot_cp2, st, nl);
                to_f32(CP3_64, o.CP3, c->tot_cp3, st, nl);
                to_f32(CP1_64, o.CP1, c->tot_cp1, st, nl);
            } else {
                for (int l : lays)
                    for (int cc = 0; cc < C; cc++) {
                        const CellDesc &cd = c->cells[c->layers[l].cell0 + cc];
                        to_f32(CP2_64 + cd.P2_off, o.CP2 + cd.P2_off, 16LL * cd.no * cd.Lt, st, nl);
                        to_f32(CP3_64 + cd.P3_off, o.CP3 + cd.P3_off, 16LL * cd.no * c->lr_r, st, nl);
                        if (cc < C - 1)
                            to_f32(CP1_64 + cd.P1_off, o.CP1 + cd.P1_off,
                                   8LL * c->lr_r * (cd.no + c->cells[c->layers[l].cell0 + cc + 1].no), st, nl);
                    }
                for (const LayerDesc &ld : lsub) {
                    const long long nlr = (long long)J * 2 * r * 2 * ld.nz, nm = (long long)J * 3 * r * r;
                    const long long nlam = (long long)(2 * r * J) * (2 * r * J);
                    to_f32(STW64 + ld.lr_off, o.STW + ld.lr_off, nlr, st, nl);
                    to_f32(UX64 + ld.lr_off, o.UX + ld.lr_off, nlr, st, nl);
                    to_f32(MRN64 + ld.m_off, o.MRN + ld.m_off, nm, st, nl);
                    to_f32(LAM64 + ld.lam_off, o.LAM + ld.lam_off, nlam, st, nl);
                }
            }
        }
        if (c->opts.tensor_cores && c->max_nx <= 128) {
            // split TF32 copy of the cell blocks for the tensor-core cell solve
            if (first) {
                long long off = 0;
                for (CellDesc &cd : c->cells) {
                    cd.tc_off = off;
                    off += cell_tc_floats(cd.nx, cd.nz);
                }
                HZ_CU(cudaMemcpyAsync(c->d_cells, c->cells.data(), sizeof(CellDesc) * c->cells.size(),
                                      cudaMemcpyHostToDevice, st));
                c->wtc = (float *)c->dalloc(sizeof(float) * std::max(off, 1LL));
                build_wtc(c->d_cells, (int)c->cells.size(), cellW, c->wtc, st, nl);
            } else {
                build_wtc(d_sub, nsub, cellW, c->wtc, st, nl);  // (sub carries the cells' tc_off)
            }
        }
        HZ_CU(cudaStreamSynchronize(st));
        for (void *q : {(void *)cellW, (void *)czv, (void *)F, (void *)E, (void *)S, (void *)Wi, (void *)Pm, (void *)Vi,
                        (void *)STW64, (void *)UX64, (void *)MRN64, (void *)LAM64, (void *)CP2_64, (void *)CP3_64,
                        (void *)CP1_64})
            c->dfree(q);
    }
    c->dfree(d_info);
    c->dfree(d_sub);
    c->dfree(d_lsub);
    HZ_CU(cudaStreamSynchronize(st));
}

void factor_all(hz_ctx *c) {
    std::vector<int> all(c->L);
    for (int l = 0; l < c->L; l++) all[l] = l;
    factor_layers(c, all, true);
}

}  // namespace hz
