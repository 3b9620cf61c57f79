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
        for (void *q : {(void *)cellW, (void *)czv, (void *)F, (void *)E, (void *)S, (void *)Wi, (void *)Pm, (void *)Vi})
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
