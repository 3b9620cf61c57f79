// C ABI entry points (include/hz.h): argument checks, host/device staging,
// error capture.  The numerical work is in hz_factor.cu and hz_solve.cu.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "hz_ctx.cuh"

using hz::CudaError;
using hz::HzError;

namespace {

thread_local std::string g_err;  // errors without a context (hz_setup failures)

// flag = 1 if any of n doubles is NaN or Inf (16-byte loads, n even)
__global__ void k_finite(const double2 *a, long long n2, int *flag) {
    bool bad = false;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
        const double2 v = a[i];
        bad |= !isfinite(v.x) || !isfinite(v.y);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicExch(flag, 1);
}

// d [B][n_rec], u [B][N]: r = R u - d; adjoint source g = R^T conj(r) (g zeroed by the
// caller; a node listed twice as a receiver receives both residuals)
__global__ void k_misfit(const double2 *__restrict__ u, const double2 *__restrict__ d, const int *__restrict__ rec,
                         int n_rec, long long N, int B, double2 *r, double2 *g) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n_rec * B;
         e += (long long)gridDim.x * blockDim.x) {
        int b = (int)(e / n_rec), i = (int)(e % n_rec);
        long long gi = (long long)b * N + rec[i];
        double2 v = make_double2(u[gi].x - d[e].x, u[gi].y - d[e].y);
        r[e] = v;
        atomicAdd(&g[gi].x, v.x);
        atomicAdd(&g[gi].y, -v.y);
    }
}

// grad_i = omega^2 sum_b Re(lambda_{b,i} u_{b,i}) / (alpha_x alpha_z)_i  with lambda the
// row-scaled-form adjoint field (so lambda / (alpha_x alpha_z) solves the transposed
// Appendix A system)
__global__ void k_grad(const double2 *__restrict__ lam, const double2 *__restrict__ u, const double2 *__restrict__ ax,
                       const double2 *__restrict__ az, int NX, long long N, int B, double om2, double *grad) {
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < N; g += (long long)gridDim.x * blockDim.x) {
        double2 D = hz::operator*(ax[g % NX], az[g / NX]);
        double s = 0.0;
        for (int b = 0; b < B; b++) {
            double2 p = hz::operator*(lam[(long long)b * N + g], u[(long long)b * N + g]);
            double2 q = hz::cdiv(p, D);
            s += q.x;
        }
        grad[g] = om2 * s;
    }
}

// out = conj(a)
__global__ void k_conj(const double2 *__restrict__ a, double2 *out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = make_double2(a[i].x, -a[i].y);
}

// mu = D^{-1} lam (lam solves the row-scaled system with source conj(gu)), grad_f = conj(mu)
__global__ void k_mu_conj(const double2 *__restrict__ lam, const double2 *__restrict__ invD, long long N, int B,
                          double2 *gf) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N * B; e += (long long)gridDim.x * blockDim.x) {
        double2 mu = hz::operator*(lam[e], invD[e % N]);
        gf[e] = make_double2(mu.x, -mu.y);
    }
}

hz_status fail(hz_ctx *c, int code, const std::string &msg) {
    if (c)
        c->err = msg;
    else
        g_err = msg;
    return (hz_status)code;
}

template <class F> hz_status guarded(hz_ctx *c, F &&f) {
    try {
        return f();
    } catch (const HzError &e) {
        return fail(c, e.code, e.what);
    } catch (const CudaError &e) {
        return fail(c, HZ_ECUDA, e.what);
    } catch (const std::bad_alloc &) {
        return fail(c, HZ_ENOMEM, "host allocation failed");
    } catch (const std::exception &e) {
        return fail(c, HZ_ECUDA, e.what());
    }
}

double2 *stage(hz_ctx *c, long long n) {
    if (c->stage_n < n) {
        c->dfree(c->stage);
        c->stage = (double2 *)c->dalloc(sizeof(double2) * n);
        c->stage_n = n;
    }
    return c->stage;
}

void check_finite(hz_ctx *c, const double *a, long long n, const char *what) {
    if (!c->d_flag) c->d_flag = (int *)c->dalloc(sizeof(int));
    HZ_CU(cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->st));
    // callers pass complex arrays (n even, 16-byte aligned)
    k_finite<<<(int)std::min<long long>(4096, (n / 2 + 255) / 256 + 1), 256, 0, c->st>>>((const double2 *)a, n / 2,
                                                                                         c->d_flag);
    HZ_CU(cudaGetLastError());
    c->nl++;
    int f = 0;
    HZ_CU(cudaMemcpyAsync(&f, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    HZ_CU(cudaStreamSynchronize(c->st));
    if (f) throw HzError(HZ_EINVAL, std::string(what) + " contains NaN or Inf");
}

// copy a user array (host or device, n complex) to a device buffer
const double2 *to_dev(hz_ctx *c, const double *a, long long n, double2 *buf) {
    if (c->opts.device_ptrs) return (const double2 *)a;
    HZ_CU(cudaMemcpyAsync(buf, a, sizeof(double2) * n, cudaMemcpyHostToDevice, c->st));
    return buf;
}
void from_dev(hz_ctx *c, double *a, const double2 *buf, long long n) {
    if (c->opts.device_ptrs) return;  // written in place
    HZ_CU(cudaMemcpyAsync(a, buf, sizeof(double2) * n, cudaMemcpyDeviceToHost, c->st));
    HZ_CU(cudaStreamSynchronize(c->st));
}

}  // namespace

extern "C" {

void hz_default_opts(hz_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->precision = HZ_FP64;
    o->precond = HZ_PGS;
    o->restart = 30;
    o->max_it = 200;
    o->tol = 0.0;  // 0: precision default (1e-10 FP64, 3e-5 mixed)
    o->refine_tol = 1e-8;
    o->max_refine = 6;
    o->pml_C = 0.0;
    o->tensor_cores = 1;
    o->rhs_lanes = 1;
    o->wait_ms = 1000.0;
    o->compress = -1.0;  // automatic: 1e-8 in mixed precision, dense in FP64
}

// HZ_FAULT=alloc[:n] | singular | nan | noconv (documented in hz.h)
static void read_fault(hz_ctx *c) {
    const char *e = std::getenv("HZ_FAULT");
    if (!e || !*e) return;
    const std::string v(e);
    if (v.rfind("alloc", 0) == 0) {
        c->fault = hz_ctx::FAULT_ALLOC;
        if (v.size() > 6 && v[5] == ':') c->fault_n = std::max(1LL, std::atoll(v.c_str() + 6));
    } else if (v == "singular") {
        c->fault = hz_ctx::FAULT_SINGULAR;
    } else if (v == "nan") {
        c->fault = hz_ctx::FAULT_NAN;
    } else if (v == "noconv") {
        c->fault = hz_ctx::FAULT_NOCONV;
    }
}

hz_status hz_setup(hz_ctx **out, const double *m, int n_x, int n_z, double omega, double h, int n_pml, int L, int C,
                   const hz_opts *opts) {
    if (!out) return fail(nullptr, HZ_EINVAL, "ctx pointer is NULL");
    *out = nullptr;
    if (!m) return fail(nullptr, HZ_EINVAL, "m is NULL");
    if (n_x < 1 || n_z < 1 || n_pml < 1 || L < 2 || C < 1 || L > n_z || C > n_x)
        return fail(nullptr, HZ_EINVAL, "need n_x, n_z >= 1, n_pml >= 1, 2 <= L <= n_z, 1 <= C <= n_x");
    if (!(std::isfinite(omega) && omega > 0 && std::isfinite(h) && h > 0))
        return fail(nullptr, HZ_EINVAL, "omega and h must be finite and positive");
    hz_ctx *c = new (std::nothrow) hz_ctx();
    if (!c) return fail(nullptr, HZ_ENOMEM, "host allocation failed");
    hz_default_opts(&c->opts);
    if (opts) c->opts = *opts;
    if (!(c->opts.wait_ms > 0)) c->opts.wait_ms = 1000.0;
    read_fault(c);
    if (c->opts.restart < 1) c->opts.restart = 30;
    if (c->opts.max_it < 1) c->opts.max_it = 200;
    // mixed: the first pass only has to bring the volume residual near the FP32
    // operators' accuracy, the refinement passes carry it to refine_tol
    if (c->opts.tol <= 0) c->opts.tol = c->opts.precision == HZ_MIXED ? 3e-5 : 1e-10;
    if (c->opts.precision != HZ_FP64 && c->opts.precision != HZ_MIXED) {
        delete c;
        return fail(nullptr, HZ_EINVAL, "precision must be HZ_FP64 or HZ_MIXED");
    }
    if (c->opts.precond < HZ_PGS || c->opts.precond > HZ_PNONE) {
        delete c;
        return fail(nullptr, HZ_EINVAL, "precond must be HZ_PGS, HZ_PJAC or HZ_PNONE");
    }
    if (c->opts.krylov != HZ_GMRES && c->opts.krylov != HZ_BICGSTAB) {
        delete c;
        return fail(nullptr, HZ_EINVAL, "krylov must be HZ_GMRES or HZ_BICGSTAB");
    }
    if (c->opts.rhs_lanes < 1 || c->opts.rhs_lanes > 8) {
        delete c;
        return fail(nullptr, HZ_EINVAL, "rhs_lanes must be 1..8");
    }
    if (c->opts.tensor_cores < 0 || c->opts.tensor_cores > 2) {
        delete c;
        return fail(nullptr, HZ_EINVAL, "tensor_cores must be 0, 1 or 2");
    }
    if (c->opts.inner != HZ_INNER_LU && c->opts.inner != HZ_INNER_NESTED) {
        delete c;
        return fail(nullptr, HZ_EINVAL, "inner must be HZ_INNER_LU or HZ_INNER_NESTED");
    }
    if (c->opts.inner == HZ_INNER_NESTED && (C < 2 || c->opts.krylov != HZ_GMRES || c->opts.rhs_lanes != 1)) {
        delete c;
        return fail(nullptr, HZ_EINVAL, "inner HZ_INNER_NESTED needs C >= 2, krylov HZ_GMRES and rhs_lanes 1");
    }
    if (!(c->opts.inner_tol > 0)) c->opts.inner_tol = 1e-6;
    if (c->opts.compress < 0) c->opts.compress = c->opts.precision == HZ_MIXED ? 1e-8 : 0.0;
    if (!(c->opts.compress >= 0) || c->opts.compress >= 1) {
        delete c;
        return fail(nullptr, HZ_EINVAL, "compress must be 0 (dense) or a tolerance in (0, 1)");
    }
    c->n_x = n_x;
    c->n_z = n_z;
    c->p = n_pml;
    c->L = L;
    c->C = C;
    c->omega = omega;
    c->h = h;
    c->NX = n_x + 2 * n_pml;
    c->NZ = n_z + 2 * n_pml;
    c->st = (cudaStream_t)c->opts.stream;
    if (cudaGetDevice(&c->dev) != cudaSuccess) c->dev = -1;
    const long long N = (long long)c->NX * c->NZ;
    double cmax = 0;
    for (long long i = 0; i < N; i++) {
        if (!std::isfinite(m[i]) || m[i] <= 0) {
            delete c;
            return fail(nullptr, HZ_EINVAL, "m must be finite and positive");
        }
        cmax = std::max(cmax, 1.0 / std::sqrt(m[i]));
    }
    c->pml_C = c->opts.pml_C > 0 ? c->opts.pml_C : 1.5 * cmax * std::log(1e6);
    auto part = [](const int *a, int parts, int n, std::vector<int> &v) {
        v.resize(parts);
        if (!a) {
            for (int i = 0; i < parts; i++) v[i] = n / parts + (i < n % parts ? 1 : 0);
            return true;
        }
        long long s = 0;
        for (int i = 0; i < parts; i++) {
            if (a[i] < 1) return false;
            v[i] = a[i];
            s += a[i];
        }
        return s == n;
    };
    if (!part(c->opts.layer_rows, L, n_z, c->rows) || !part(c->opts.cell_cols, C, n_x, c->cols)) {
        delete c;
        return fail(nullptr, HZ_EINVAL, "layer_rows must be L positive counts summing to n_z, cell_cols C summing to n_x");
    }
    c->opts.layer_rows = nullptr;  // copied
    c->opts.cell_cols = nullptr;
    hz_status s = guarded(c, [&]() -> hz_status {
        c->d_m = (double *)c->dalloc(sizeof(double) * N);
        HZ_CU(cudaMemcpy(c->d_m, m, sizeof(double) * N, cudaMemcpyHostToDevice));
        c->h_m.assign(m, m + N);
        hz::build_decomposition(c);
        hz::init_global_alpha(c);
        return HZ_OK;
    });
    if (s != HZ_OK) {
        g_err = c->err;
        hz_destroy(c);
        return s;
    }
    *out = c;
    return HZ_OK;
}

// Inner nested level (opts.inner = HZ_INNER_NESTED, Section 4.2): per layer, a
// context of the layer's box with x and z swapped -- the layer's medium with
// its artificial PML rows extending its first / last row, transposed; its
// layers are the cells (one cell each) -- factored, with a lane for 2B-wide
// applications.
static void build_inner(hz_ctx *c) {
    const int L = c->L, p = c->p, NX = c->NX;
    for (hz_ctx *ic : c->inner_ctx) hz_destroy(ic);  // a failed earlier attempt
    c->inner_ctx.assign(L, nullptr);
    c->inner_wide.assign(L, nullptr);
    for (int l = 0; l < L; l++) {
        const hz::LayerDesc &ld = c->layers[l];
        const int nz = ld.nz, n = ld.n;
        std::vector<double> mt((size_t)NX * nz);
        for (int r = 0; r < nz; r++) {
            int g = ld.s + r;  // global array row of local row r
            if (l > 0) g = std::max(g, ld.s + p);
            if (l < L - 1) g = std::min(g, ld.s + n + p - 1);
            for (int x = 0; x < NX; x++) mt[(size_t)x * nz + r] = c->h_m[(size_t)g * NX + x];
        }
        hz_opts io;
        hz_default_opts(&io);
        io.precision = c->opts.precision;
        io.precond = HZ_PGS;
        io.max_it = 60;
        io.tol = c->opts.inner_tol;
        io.refine_tol = 0.0;
        io.max_refine = 1;
        io.pml_C = c->pml_C;
        io.layer_rows = c->cols.data();
        io.device_ptrs = 1;
        io.tensor_cores = c->opts.tensor_cores;
        io.wait_ms = c->opts.wait_ms;
        cudaStream_t s = nullptr;
        HZ_CU(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        io.stream = s;
        hz_ctx *ic = nullptr;
        hz_status st = hz_setup(&ic, mt.data(), n, c->n_x, c->omega, c->h, p, c->C, 1, &io);
        if (st != HZ_OK) {
            cudaStreamDestroy(s);
            throw HzError(st, std::string("inner context of a layer: ") + hz_last_error(nullptr));
        }
        ic->own_stream = true;
        c->inner_ctx[l] = ic;
        st = hz_factor(ic);
        if (st != HZ_OK) throw HzError(st, "inner context of a layer: " + ic->err);
        hz_ctx *w = hz::make_lane(ic);
        ic->lanes.push_back(w);
        c->inner_wide[l] = w;
    }
}

hz_status hz_factor(hz_ctx *c) {
    if (!c) return fail(nullptr, HZ_EINVAL, "ctx is NULL");
    if (c->factored) return HZ_OK;
    c->nl = 0;
    return guarded(c, [&]() -> hz_status {
        hz::factor_all(c);
        if (c->nested()) build_inner(c);
        c->factored = true;
        return HZ_OK;
    });
}

hz_status hz_update_model(hz_ctx *c, const double *m_new, int *n_layers) {
    if (!c) return fail(nullptr, HZ_EINVAL, "ctx is NULL");
    if (!m_new) return fail(c, HZ_EINVAL, "m_new must be non-NULL");
    if (!c->factored) return fail(c, HZ_ESTATE, "hz_update_model before hz_factor");
    if (c->nested()) return fail(c, HZ_EINVAL, "hz_update_model is not available with the nested inner level");
    const int NX = c->NX, NZ = c->NZ;
    const long long N = (long long)NX * NZ;
    for (long long i = 0; i < N; i++)
        if (!std::isfinite(m_new[i]) || m_new[i] <= 0) return fail(c, HZ_EINVAL, "m_new must be finite and positive");
    c->nl = 0;
    return guarded(c, [&]() -> hz_status {
        // changed points, as a 2D prefix count: a cell is touched when its read box holds one
        std::vector<long long> cnt((size_t)(NZ + 1) * (NX + 1), 0);
        long long changed = 0;
        for (int z = 0; z < NZ; z++)
            for (int x = 0; x < NX; x++) {
                const int d = m_new[(long long)z * NX + x] != c->h_m[(long long)z * NX + x];
                changed += d;
                cnt[(size_t)(z + 1) * (NX + 1) + x + 1] = d + cnt[(size_t)z * (NX + 1) + x + 1] +
                                                          cnt[(size_t)(z + 1) * (NX + 1) + x] - cnt[(size_t)z * (NX + 1) + x];
            }
        auto box = [&](int z0, int z1, int x0, int x1) {  // changed points in rows [z0, z1], columns [x0, x1]
            return cnt[(size_t)(z1 + 1) * (NX + 1) + x1 + 1] - cnt[(size_t)z0 * (NX + 1) + x1 + 1] -
                   cnt[(size_t)(z1 + 1) * (NX + 1) + x0] + cnt[(size_t)z0 * (NX + 1) + x0];
        };
        std::vector<int> lays;
        if (changed) {
            const int p = c->p;
            for (int l = 0; l < c->L; l++) {
                bool touched = false;
                for (int cc = 0; cc < c->C && !touched; cc++) {
                    // the grid points the cell's coefficients read (its box, with the
                    // neighbour sides clamped to the interior as in the coefficient kernel)
                    const hz::CellDesc &cd = c->cells[c->layers[l].cell0 + cc];
                    const int z0 = cd.top ? cd.s + p : cd.s, z1 = cd.bot ? cd.s + cd.n + p - 1 : cd.s + cd.nz - 1;
                    const int x0 = cd.left ? cd.t + p : cd.t, x1 = cd.right ? cd.t + cd.w + p - 1 : cd.t + cd.nx - 1;
                    touched = box(z0, z1, x0, x1) > 0;
                }
                if (touched) lays.push_back(l);
            }
            HZ_CU(cudaMemcpy(c->d_m, m_new, sizeof(double) * N, cudaMemcpyHostToDevice));
            c->h_m.assign(m_new, m_new + N);
            hz::launch_cell_coeffs(c->d_gcell, 1, c->d_m, NX, c->omega, c->h, c->pml_C, c->p, c->d_gdiag, c->d_gcx,
                                   c->d_gcz, c->st, &c->nl);
            hz::factor_layers(c, lays, false);
            if (c->mixed() && c->opts.tensor_cores == 2) hz::tc_refresh_operators(c);
            HZ_CU(cudaStreamSynchronize(c->st));
        }
        if (n_layers) *n_layers = (int)lays.size();
        return HZ_OK;
    });
}

hz_status hz_solve(hz_ctx *c, const double *f, int B, double *u, hz_stats *st) {
    if (!c) return fail(nullptr, HZ_EINVAL, "ctx is NULL");
    if (!c->factored) return fail(c, HZ_ESTATE, "hz_solve before hz_factor");
    if (!f || !u || B < 1) return fail(c, HZ_EINVAL, "f, u must be non-NULL and B >= 1");
    c->nl = 0;
    return guarded(c, [&]() -> hz_status {
        const long long N = (long long)c->NX * c->NZ;
        double2 *buf = stage(c, 2 * N * B);
        const double2 *fd = to_dev(c, f, N * B, buf);
        check_finite(c, (const double *)fd, 2 * N * B, "f");
        double2 *ud = c->opts.device_ptrs ? (double2 *)u : buf + N * B;
        c->kt_reset();
        int s = c->mixed() ? hz::solve_impl<float2>(c, fd, B, ud, st, true)
                           : hz::solve_impl<double2>(c, fd, B, ud, st, true);
        from_dev(c, u, ud, N * B);
        c->kt_collect();
        if (st) {
            st->gpu_launches = c->nl;
            for (int i = 0; i < 3; i++) {
                st->kt_launches[i] = c->kt_launches[i];
                st->kt_ms[i] = c->kt_ms[i];
                st->kt_bytes[i] = c->kt_bytes[i];
                st->kt_flops[i] = c->kt_flops[i];
            }
        }
        if (s == HZ_ENOTCONV) c->err = "tolerance not reached; best iterate written";
        return (hz_status)s;
    });
}

hz_status hz_solve_group(hz_ctx **cs, int G, const double *const *f, int B, double *const *u, hz_stats *st) {
    if (!cs || G < 1) return fail(nullptr, HZ_EINVAL, "ctxs must be non-NULL and G >= 1");
    for (int i = 0; i < G; i++)
        if (!cs[i]) return fail(nullptr, HZ_EINVAL, "a ctx in the group is NULL");
    hz_ctx *c0 = cs[0];
    if (!f || !u || B < 1) return fail(c0, HZ_EINVAL, "f, u must be non-NULL and B >= 1");
    int dev0 = c0->dev;
    for (int i = 0; i < G; i++) {
        if (!cs[i]->factored) return fail(c0, HZ_ESTATE, "hz_solve_group before hz_factor on every member");
        if (cs[i]->mixed() != c0->mixed()) return fail(c0, HZ_EINVAL, "group members must share the precision");
        if (cs[i]->opts.krylov != c0->opts.krylov)
            return fail(c0, HZ_EINVAL, "group members must share the Krylov method");
        if (cs[i]->dev != dev0) return fail(c0, HZ_EINVAL, "group members must share the device");
        if (!f[i] || !u[i]) return fail(c0, HZ_EINVAL, "f[i], u[i] must be non-NULL");
        for (int j = 0; j < i; j++)
            if (cs[j] == cs[i]) return fail(c0, HZ_EINVAL, "a ctx appears twice in the group");
    }
    for (int i = 0; i < G; i++) cs[i]->nl = 0;
    return guarded(c0, [&]() -> hz_status {
        std::vector<hz_ctx *> v(cs, cs + G);
        std::vector<const double2 *> fd(G);
        std::vector<double2 *> ud(G);
        for (int i = 0; i < G; i++) {
            hz_ctx *c = cs[i];
            const long long N = (long long)c->NX * c->NZ;
            double2 *buf = stage(c, 2 * N * B);
            fd[i] = to_dev(c, f[i], N * B, buf);
            check_finite(c, (const double *)fd[i], 2 * N * B, "f");
            ud[i] = c->opts.device_ptrs ? (double2 *)u[i] : buf + N * B;
            c->kt_reset();
        }
        std::vector<hz_stats> sts;
        int s = c0->mixed() ? hz::solve_group_impl<float2>(v, fd, B, ud, sts, true)
                            : hz::solve_group_impl<double2>(v, fd, B, ud, sts, true);
        for (int i = 0; i < G; i++) {
            hz_ctx *c = cs[i];
            from_dev(c, u[i], ud[i], (long long)c->NX * c->NZ * B);
            c->kt_collect();
            if (st) {
                st[i] = sts[i];
                st[i].gpu_launches = c->nl;
                for (int k = 0; k < 3; k++) {
                    st[i].kt_launches[k] = c->kt_launches[k];
                    st[i].kt_ms[k] = c->kt_ms[k];
                    st[i].kt_bytes[k] = c->kt_bytes[k];
                    st[i].kt_flops[k] = c->kt_flops[k];
                }
            }
        }
        if (s == HZ_ENOTCONV) c0->err = "tolerance not reached by a group member; best iterates written";
        return (hz_status)s;
    });
}

hz_status hz_gradient(hz_ctx *c, const double *f, int B, const double *d, const int *rec_idx, int n_rec, double *J,
                      double *grad_m, double *u_out, hz_stats *st) {
    if (!c) return fail(nullptr, HZ_EINVAL, "ctx is NULL");
    if (!c->factored) return fail(c, HZ_ESTATE, "hz_gradient before hz_factor");
    if (!f || !d || !rec_idx || n_rec < 1 || !J || !grad_m || B < 1)
        return fail(c, HZ_EINVAL, "NULL argument or n_rec < 1 or B < 1");
    c->nl = 0;
    return guarded(c, [&]() -> hz_status {
        const long long N = (long long)c->NX * c->NZ;
        cudaStream_t s_ = c->st;
        // device buffers: f/u (2NB) staging + lambda, g, r, d, rec, grad
        double2 *buf = stage(c, 2 * N * B);
        const double2 *fd = to_dev(c, f, N * B, buf);
        check_finite(c, (const double *)fd, 2 * N * B, "f");
        double2 *ud = buf + N * B;
        double2 *g = (double2 *)c->dalloc(sizeof(double2) * N * B);
        double2 *lam = (double2 *)c->dalloc(sizeof(double2) * N * B);
        double2 *r = (double2 *)c->dalloc(sizeof(double2) * (long long)n_rec * B);
        double2 *dd = (double2 *)c->dalloc(sizeof(double2) * (long long)n_rec * B);
        int *rd = (int *)c->dalloc(sizeof(int) * n_rec);
        double *gd = (double *)c->dalloc(sizeof(double) * N);
        struct Free {
            hz_ctx *c;
            std::vector<void *> v;
            ~Free() {
                for (void *p : v) c->dfree(p);
            }
        } fr{c, {g, lam, r, dd, rd, gd}};
        // the receiver indices are range-checked on the host in both pointer modes (a
        // device list is read back first: the kernel indexes u and g with them)
        std::vector<int> rh_idx((size_t)n_rec);
        if (c->opts.device_ptrs) {
            HZ_CU(cudaMemcpyAsync(rh_idx.data(), rec_idx, sizeof(int) * n_rec, cudaMemcpyDeviceToHost, s_));
            HZ_CU(cudaStreamSynchronize(s_));
        } else {
            std::memcpy(rh_idx.data(), rec_idx, sizeof(int) * n_rec);
        }
        for (int i = 0; i < n_rec; i++)
            if (rh_idx[i] < 0 || rh_idx[i] >= N) throw HzError(HZ_EINVAL, "receiver index out of range");
        HZ_CU(cudaMemcpyAsync(dd, d, sizeof(double2) * (long long)n_rec * B,
                              c->opts.device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s_));
        HZ_CU(cudaMemcpyAsync(rd, rh_idx.data(), sizeof(int) * n_rec, cudaMemcpyHostToDevice, s_));
        HZ_CU(cudaStreamSynchronize(s_));  // rh_idx is a pageable host vector
        hz_stats s1{}, s2{};
        c->kt_reset();
        int sf = c->mixed() ? hz::solve_impl<float2>(c, fd, B, ud, &s1, true)
                            : hz::solve_impl<double2>(c, fd, B, ud, &s1, true);
        HZ_CU(cudaMemsetAsync(g, 0, sizeof(double2) * N * B, s_));
        k_misfit<<<256, 256, 0, s_>>>(ud, dd, rd, n_rec, N, B, r, g);
        HZ_CU(cudaGetLastError());
        c->nl++;
        std::vector<double2> rh((size_t)n_rec * B);
        HZ_CU(cudaMemcpyAsync(rh.data(), r, sizeof(double2) * rh.size(), cudaMemcpyDeviceToHost, s_));
        HZ_CU(cudaStreamSynchronize(s_));
        double Jv = 0;
        for (auto &v : rh) Jv += v.x * v.x + v.y * v.y;
        *J = 0.5 * Jv;
        // adjoint: the row-scaled operator is symmetric, so the same factors solve it
        int sa = c->mixed() ? hz::solve_impl<float2>(c, g, B, lam, &s2, false)
                            : hz::solve_impl<double2>(c, g, B, lam, &s2, false);
        k_grad<<<256, 256, 0, s_>>>(lam, ud, c->d_ax, c->d_az, c->NX, N, B, c->omega * c->omega, gd);
        HZ_CU(cudaGetLastError());
        c->nl++;
        if (c->opts.device_ptrs) {
            HZ_CU(cudaMemcpyAsync(grad_m, gd, sizeof(double) * N, cudaMemcpyDeviceToDevice, s_));
            if (u_out) HZ_CU(cudaMemcpyAsync(u_out, ud, sizeof(double2) * N * B, cudaMemcpyDeviceToDevice, s_));
        } else {
            HZ_CU(cudaMemcpyAsync(grad_m, gd, sizeof(double) * N, cudaMemcpyDeviceToHost, s_));
            if (u_out) HZ_CU(cudaMemcpyAsync(u_out, ud, sizeof(double2) * N * B, cudaMemcpyDeviceToHost, s_));
        }
        HZ_CU(cudaStreamSynchronize(s_));
        if (st) {
            *st = s1;
            st->iterations += s2.iterations;
            st->refinements += s2.refinements;
            st->resid = std::max(s1.resid, s2.resid);
            st->t_total_ms += s2.t_total_ms;
            st->t_local_ms += s2.t_local_ms;
            st->t_gmres_ms += s2.t_gmres_ms;
            st->t_recon_ms += s2.t_recon_ms;
            st->t_resid_ms += s2.t_resid_ms;
            st->gpu_launches = c->nl;
            c->kt_collect();
            for (int i = 0; i < 3; i++) {
                st->kt_launches[i] = c->kt_launches[i];
                st->kt_ms[i] = c->kt_ms[i];
                st->kt_bytes[i] = c->kt_bytes[i];
                st->kt_flops[i] = c->kt_flops[i];
            }
        }
        return (hz_status)(sf != HZ_OK ? sf : sa);
    });
}

hz_status hz_adjoint(hz_ctx *c, const double *u, const double *gu, int B, double *grad_m, double *grad_f,
                     hz_stats *st) {
    if (!c) return fail(nullptr, HZ_EINVAL, "ctx is NULL");
    if (!c->factored) return fail(c, HZ_ESTATE, "hz_adjoint before hz_factor");
    if (!u || !gu || !grad_m || B < 1) return fail(c, HZ_EINVAL, "NULL argument or B < 1");
    c->nl = 0;
    return guarded(c, [&]() -> hz_status {
        const long long N = (long long)c->NX * c->NZ;
        cudaStream_t s_ = c->st;
        double2 *buf = stage(c, 2 * N * B);
        const double2 *ud = to_dev(c, u, N * B, buf);
        double2 *gbuf = (double2 *)c->dalloc(sizeof(double2) * N * B);
        double2 *lam = (double2 *)c->dalloc(sizeof(double2) * N * B);
        double *gd = (double *)c->dalloc(sizeof(double) * N);
        struct Free {
            hz_ctx *c;
            std::vector<void *> v;
            ~Free() {
                for (void *p : v) c->dfree(p);
            }
        } fr{c, {gbuf, lam, gd}};
        const double2 *gud = to_dev(c, gu, N * B, buf + N * B);
        check_finite(c, (const double *)gud, 2 * N * B, "gu");
        k_conj<<<256, 256, 0, s_>>>(gud, gbuf, N * B);
        HZ_CU(cudaGetLastError());
        c->nl++;
        c->kt_reset();
        hz_stats s1{};
        // H^T = (D H_s)^T = H_s D: mu = D^{-1} H_s^{-1} conj(gu); the symmetric solve takes
        // conj(gu) as its row-scaled source directly
        int sa = c->mixed() ? hz::solve_impl<float2>(c, gbuf, B, lam, &s1, false)
                            : hz::solve_impl<double2>(c, gbuf, B, lam, &s1, false);
        k_grad<<<256, 256, 0, s_>>>(lam, ud, c->d_ax, c->d_az, c->NX, N, B, c->omega * c->omega, gd);
        HZ_CU(cudaGetLastError());
        c->nl++;
        if (grad_f) {
            double2 *gfd = c->opts.device_ptrs ? (double2 *)grad_f : gbuf;  // gbuf no longer needed
            k_mu_conj<<<256, 256, 0, s_>>>(lam, c->d_ginvD, N, B, gfd);
            HZ_CU(cudaGetLastError());
            c->nl++;
            if (!c->opts.device_ptrs)
                HZ_CU(cudaMemcpyAsync(grad_f, gfd, sizeof(double2) * N * B, cudaMemcpyDeviceToHost, s_));
        }
        if (c->opts.device_ptrs)
            HZ_CU(cudaMemcpyAsync(grad_m, gd, sizeof(double) * N, cudaMemcpyDeviceToDevice, s_));
        else
            HZ_CU(cudaMemcpyAsync(grad_m, gd, sizeof(double) * N, cudaMemcpyDeviceToHost, s_));
        HZ_CU(cudaStreamSynchronize(s_));
        c->kt_collect();
        if (st) {
            *st = s1;
            st->gpu_launches = c->nl;
        }
        return (hz_status)sa;
    });
}

hz_status hz_cell_solve(hz_ctx *c, int l, int cc, const double *g, int B, double *x) {
    if (!c) return fail(nullptr, HZ_EINVAL, "ctx is NULL");
    if (!c->factored) return fail(c, HZ_ESTATE, "hz_cell_solve before hz_factor");
    if (l < 0 || l >= c->L || cc < 0 || cc >= c->C || !g || !x || B < 1) return fail(c, HZ_EINVAL, "bad argument");
    c->nl = 0;
    return guarded(c, [&]() -> hz_status {
        const int ci = l * c->C + cc;
        const long long n = (long long)c->cells[ci].nx * c->cells[ci].nz;
        double2 *buf = stage(c, 2 * n * B);
        const double2 *gd = to_dev(c, g, n * B, buf);
        double2 *xd = c->opts.device_ptrs ? (double2 *)x : buf + n * B;
        if (c->mixed())
            hz::comp_cell_solve<float2>(c, ci, gd, B, xd);
        else
            hz::comp_cell_solve<double2>(c, ci, gd, B, xd);
        from_dev(c, x, xd, n * B);
        return HZ_OK;
    });
}

hz_status hz_layer_green(hz_ctx *c, int l, const double *tr, int in_mask, int B, double *out) {
    if (!c) return fail(nullptr, HZ_EINVAL, "ctx is NULL");
    if (!c->factored) return fail(c, HZ_ESTATE, "hz_layer_green before hz_factor");
    if (l < 0 || l >= c->L || !tr || !out || B < 1 || in_mask < 0 || in_mask > 3)
        return fail(c, HZ_EINVAL, "bad argument");
    c->nl = 0;
    return guarded(c, [&]() -> hz_status {
        const long long n = 4LL * c->NX;
        double2 *buf = stage(c, 2 * n * B);
        const double2 *td = to_dev(c, tr, n * B, buf);
        double2 *od = c->opts.device_ptrs ? (double2 *)out : buf + n * B;
        if (c->mixed())
            hz::comp_layer_green<float2>(c, l, td, in_mask, B, od);
        else
            hz::comp_layer_green<double2>(c, l, td, in_mask, B, od);
        from_dev(c, out, od, n * B);
        return HZ_OK;
    });
}

static hz_status polar(hz_ctx *c, int which, const double *x, int B, double *y) {
    if (!c) return fail(nullptr, HZ_EINVAL, "ctx is NULL");
    if (!c->factored) return fail(c, HZ_ESTATE, "called before hz_factor");
    if (!x || !y || B < 1 || which < -1 || which > 4) return fail(c, HZ_EINVAL, "bad argument");
    c->nl = 0;
    return guarded(c, [&]() -> hz_status {
        const long long n = c->n_tr();
        double2 *buf = stage(c, 2 * n * B);
        const double2 *xd = to_dev(c, x, n * B, buf);
        double2 *yd = c->opts.device_ptrs ? (double2 *)y : buf + n * B;
        if (c->mixed())
            hz::comp_polar<float2>(c, which, xd, B, yd);
        else
            hz::comp_polar<double2>(c, which, xd, B, yd);
        from_dev(c, y, yd, n * B);
        return HZ_OK;
    });
}

hz_status hz_apply_M(hz_ctx *c, const double *x, int B, double *y) { return polar(c, -1, x, B, y); }
hz_status hz_precond(hz_ctx *c, int which, const double *x, int B, double *y) {
    if (which < 0) return fail(c, HZ_EINVAL, "which must be 0..4");
    return polar(c, which, x, B, y);
}

hz_status hz_residual(hz_ctx *c, const double *u, const double *f, int B, double *res) {
    if (!c) return fail(nullptr, HZ_EINVAL, "ctx is NULL");
    if (!u || !f || !res || B < 1) return fail(c, HZ_EINVAL, "bad argument");
    c->nl = 0;
    return guarded(c, [&]() -> hz_status {
        const long long N = (long long)c->NX * c->NZ;
        double2 *buf = stage(c, 2 * N * B);
        const double2 *ud = c->opts.device_ptrs ? (const double2 *)u : buf;
        const double2 *fd = c->opts.device_ptrs ? (const double2 *)f : buf + N * B;
        if (!c->opts.device_ptrs) {
            HZ_CU(cudaMemcpyAsync(buf, u, sizeof(double2) * N * B, cudaMemcpyHostToDevice, c->st));
            HZ_CU(cudaMemcpyAsync(buf + N * B, f, sizeof(double2) * N * B, cudaMemcpyHostToDevice, c->st));
        }
        std::vector<double> r(B);
        if (c->mixed())
            hz::comp_residual<float2>(c, ud, fd, B, r.data());
        else
            hz::comp_residual<double2>(c, ud, fd, B, r.data());
        if (c->opts.device_ptrs)
            HZ_CU(cudaMemcpy(res, r.data(), sizeof(double) * B, cudaMemcpyHostToDevice));
        else
            std::memcpy(res, r.data(), sizeof(double) * B);
        return HZ_OK;
    });
}

hz_status hz_traces(hz_ctx *c, const double *u, int B, double *tr) {
    if (!c) return fail(nullptr, HZ_EINVAL, "ctx is NULL");
    if (!u || !tr || B < 1) return fail(c, HZ_EINVAL, "u, tr must be non-NULL and B >= 1");
    if (c->L < 2) return fail(c, HZ_EINVAL, "a single layer has no interface traces");
    c->nl = 0;
    return guarded(c, [&]() -> hz_status {
        const long long N = (long long)c->NX * c->NZ;
        const long long T = (long long)(c->L - 1) * 2 * c->NX * B;
        double2 *buf = stage(c, N * B + T);
        const double2 *ud = to_dev(c, u, N * B, buf);
        double2 *td = c->opts.device_ptrs ? (double2 *)tr : buf + N * B;
        hz::comp_traces(c, ud, B, td);
        from_dev(c, tr, td, T);
        if (c->opts.device_ptrs) HZ_CU(cudaStreamSynchronize(c->st));
        return HZ_OK;
    });
}

hz_status hz_reconstruct(hz_ctx *c, const double *f, const double *tr, int B, double *u) {
    if (!c) return fail(nullptr, HZ_EINVAL, "ctx is NULL");
    if (!c->factored) return fail(c, HZ_ESTATE, "hz_reconstruct before hz_factor");
    if (!f || !tr || !u || B < 1) return fail(c, HZ_EINVAL, "f, tr, u must be non-NULL and B >= 1");
    if (c->L < 2) return fail(c, HZ_EINVAL, "a single layer has no interface traces");
    c->nl = 0;
    return guarded(c, [&]() -> hz_status {
        const long long N = (long long)c->NX * c->NZ;
        const long long T = (long long)(c->L - 1) * 2 * c->NX * B;
        double2 *buf = stage(c, 2 * N * B + T);
        const double2 *fd = to_dev(c, f, N * B, buf);
        const double2 *td = c->opts.device_ptrs ? (const double2 *)tr : buf + N * B;
        if (!c->opts.device_ptrs)
            HZ_CU(cudaMemcpyAsync(buf + N * B, tr, sizeof(double2) * T, cudaMemcpyHostToDevice, c->st));
        check_finite(c, (const double *)fd, 2 * N * B, "f");
        check_finite(c, (const double *)td, 2 * T, "tr");
        double2 *ud = c->opts.device_ptrs ? (double2 *)u : buf + N * B + T;
        if (c->mixed())
            hz::comp_reconstruct<float2>(c, fd, td, B, ud);
        else
            hz::comp_reconstruct<double2>(c, fd, td, B, ud);
        from_dev(c, u, ud, N * B);
        return HZ_OK;
    });
}

hz_status hz_check_timeout(hz_ctx *c) {
    if (!c) return fail(nullptr, HZ_EINVAL, "ctx is NULL");
    return guarded(c, [&]() -> hz_status {
        c->nl = 0;
        HZ_CU(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->st));
        hz::launch_wait_check(c->d_err, c->st, &c->nl);
        int e = 0;
        HZ_CU(cudaMemcpyAsync(&e, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
        HZ_CU(cudaStreamSynchronize(c->st));
        if (!e) return HZ_OK;
        HZ_CU(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->st));
        HZ_CU(cudaStreamSynchronize(c->st));
        char b[160];
        snprintf(b, sizeof b, "a bounded device wait gave up after %.3f ms (timeout check)", c->opts.wait_ms);
        c->err = b;
        return HZ_ETIMEOUT;
    });
}

hz_status hz_set_device_ptrs(hz_ctx *c, int device_ptrs) {
    if (!c) return fail(nullptr, HZ_EINVAL, "ctx is NULL");
    c->opts.device_ptrs = device_ptrs ? 1 : 0;
    return HZ_OK;
}

hz_status hz_set_time_kernels(hz_ctx *c, int time_kernels) {
    if (!c) return fail(nullptr, HZ_EINVAL, "ctx is NULL");
    c->opts.time_kernels = time_kernels ? 1 : 0;
    return HZ_OK;
}

long long hz_device_bytes(const hz_ctx *c) {
    if (!c) return 0;
    long long b = c->dev_bytes;
    for (const hz_ctx *s : c->lanes) b += s->dev_bytes;
    return b;
}

static void destroy_one(hz_ctx *c);

void hz_destroy(hz_ctx *c) {
    if (!c) return;
    for (hz_ctx *ic : c->inner_ctx) hz_destroy(ic);  // their lanes go with them
    c->inner_ctx.clear();
    c->inner_wide.clear();
    for (hz_ctx *s : c->lanes) destroy_one(s);  // lanes own only their streams and workspaces
    c->lanes.clear();
    destroy_one(c);
}

static void destroy_one(hz_ctx *c) {
    for (auto &kv : c->allocs) cudaFree(kv.first);
    c->kt_open.clear();
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    c->ev_pool.clear();
    c->allocs.clear();
    if (c->w64) {
        if (c->w64->hhost) cudaFreeHost(c->w64->hhost);
        if (c->w64->rhost) cudaFreeHost(c->w64->rhost);
    }
    if (c->w32) {
        if (c->w32->hhost) cudaFreeHost(c->w32->hhost);
        if (c->w32->rhost) cudaFreeHost(c->w32->rhost);
    }
    if (c->own_stream && c->st) cudaStreamDestroy(c->st);
    delete c;
}

const char *hz_last_error(const hz_ctx *c) { return c ? c->err.c_str() : g_err.c_str(); }

}  // extern "C"
