// Allocation-free relative residual ||H u - f|| / ||f|| (one extra entry point).
//
// Some callers cannot call cudaMalloc at the point where they need a residual:
// a process whose device memory is fully reserved up front by another
// allocator (a framework's caching pool, a fixed arena planned at start-up),
// or a latency-critical loop that forbids allocation calls because they
// synchronise the device and may fail under memory pressure.  hz_residual
// allocates its staging and reduction buffers on first use; this variant
// keeps its only scratch (per-chunk partial sums) in a fixed file-scope
// device array instead, and reads the caller's device arrays in place.
#include <mutex>

#include "hz_ctx.cuh"

namespace {

// Maximum right-hand sides per call and partial sums per right-hand side.
constexpr int NA_MAX_B = 256;
constexpr int NA_CHUNKS = 128;

// Scratch: [NA_CHUNKS][NA_MAX_B][2] doubles = 512 KiB, held by every GPU that
// loads the library until the process exits.  Shared by all calls: each call
// writes every slot it later reads, so no clearing is needed, and calls whose
// kernels overlap on the GPU (different streams, or contexts used from
// several threads) race on it.
__device__ __align__(256) double g_na_scratch[NA_CHUNKS * NA_MAX_B * 2];

// Host-side device addresses of the scratch array, one per device.  The
// symbol's name in host code is only a host stand-in, so the address is
// looked up once per device with cudaGetSymbolAddress while that device is
// current.
constexpr int NA_MAX_DEV = 64;
std::mutex g_na_mu;
double *g_na_ptr[NA_MAX_DEV] = {};

// partial sums of |r|^2 and |f|^2 with r = f - H u (Appendix A operator, here
// alpha_x alpha_z times the row-scaled stencil), u and f batch-outer [B][N]
__global__ void __launch_bounds__(256) k_na_resid(const double2 *__restrict__ u, const double2 *__restrict__ f,
                                                  const double *__restrict__ m, const double2 *__restrict__ ax,
                                                  const double2 *__restrict__ axh, const double2 *__restrict__ az,
                                                  const double2 *__restrict__ azh, int NX, int NZ, double h,
                                                  double omega, double *part) {
    const int chunk = blockIdx.x, b = blockIdx.y, B = gridDim.y;
    const long long N = (long long)NX * NZ;
    const long long len = (N + NA_CHUNKS - 1) / NA_CHUNKS;
    const long long g0 = chunk * len, g1 = min(N, g0 + len);
    const double2 *ub = u + (long long)b * N;
    const double2 *fb = f + (long long)b * N;
    const double ih2 = 1.0 / (h * h);
    double rr = 0.0, ff = 0.0;
    for (long long g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
        const int iz = (int)(g / NX), ix = (int)(g % NX);
        const double2 a_x = ax[ix], a_z = az[iz];
        const double2 D = hz::operator*(a_x, a_z);
        const double2 cxp = hz::cdiv(axh[ix + 1], a_z), cxm = hz::cdiv(axh[ix], a_z);
        const double2 czp = hz::cdiv(azh[iz + 1], a_x), czm = hz::cdiv(azh[iz], a_x);
        const double2 uc = ub[g];
        double2 Hu = hz::operator*(hz::operator+(hz::operator+(cxp, cxm), hz::operator+(czp, czm)), uc);
        if (ix > 0) Hu = hz::operator-(Hu, hz::operator*(cxm, ub[g - 1]));
        if (ix < NX - 1) Hu = hz::operator-(Hu, hz::operator*(cxp, ub[g + 1]));
        if (iz > 0) Hu = hz::operator-(Hu, hz::operator*(czm, ub[g - NX]));
        if (iz < NZ - 1) Hu = hz::operator-(Hu, hz::operator*(czp, ub[g + NX]));
        Hu = hz::operator-(hz::operator*(ih2, Hu),
                           hz::operator*(hz::cdiv(make_double2(omega * omega * m[g], 0.0), D), uc));
        const double2 r = hz::operator-(fb[g], hz::operator*(D, Hu));
        rr += hz::cabs2(r);
        ff += hz::cabs2(fb[g]);
    }
    __shared__ double s_r[8], s_f[8];
    for (int o = 16; o > 0; o >>= 1) {
        rr += __shfl_down_sync(0xffffffffu, rr, o);
        ff += __shfl_down_sync(0xffffffffu, ff, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s_r[threadIdx.x >> 5] = rr;
        s_f[threadIdx.x >> 5] = ff;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, c = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            a += s_r[w];
            c += s_f[w];
        }
        part[((long long)chunk * B + b) * 2 + 0] = a;
        part[((long long)chunk * B + b) * 2 + 1] = c;
    }
}

__global__ void k_na_final(const double *__restrict__ part, int B, double *res) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    double a = 0, c = 0;
    for (int k = 0; k < NA_CHUNKS; k++) {
        a += part[((long long)k * B + b) * 2 + 0];
        c += part[((long long)k * B + b) * 2 + 1];
    }
    res[b] = c > 0 ? sqrt(a) / sqrt(c) : 0.0;
}

}  // namespace

extern "C" hz_status hz_residual_noalloc(hz_ctx *c, const double *u, const double *f, int B, double *res) {
    if (!c) return HZ_EINVAL;
    if (!u || !f || !res) {
        c->err = "hz_residual_noalloc: u, f and res must be device pointers";
        return HZ_EINVAL;
    }
    if (B < 1 || B > NA_MAX_B) {
        c->err = "hz_residual_noalloc: B must be in 1..256 (size of the preallocated scratch)";
        return HZ_EINVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        c->err = std::string("hz_residual_noalloc: cudaGetDevice failed: ") + cudaGetErrorString(e);
        return HZ_ECUDA;
    }
    if (dev != c->dev) {
        c->err = "hz_residual_noalloc: the current device (" + std::to_string(dev) +
                 ") is not the context's device (" + std::to_string(c->dev) + "); make it current first";
        return HZ_EINVAL;
    }
    if (dev < 0 || dev >= NA_MAX_DEV) {
        c->err = "hz_residual_noalloc: device ordinal " + std::to_string(dev) + " is beyond the " +
                 std::to_string(NA_MAX_DEV) + " devices this entry point serves";
        return HZ_EINVAL;
    }
    // u, f and res must be memory of this device (a host address would be
    // dereferenced by the kernel)
    const void *args[3] = {u, f, res};
    for (const void *a : args) {
        cudaPointerAttributes pa{};
        e = cudaPointerGetAttributes(&pa, a);
        if (e != cudaSuccess || pa.type != cudaMemoryTypeDevice || pa.device != dev) {
            (void)cudaGetLastError();  // clear a sticky-free error of the query
            c->err = "hz_residual_noalloc: u, f and res must be device memory of the context's device";
            return HZ_EINVAL;
        }
    }
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        if (!g_na_ptr[dev]) {
            e = cudaGetSymbolAddress((void **)&g_na_ptr[dev], g_na_scratch);
            if (e != cudaSuccess) {
                g_na_ptr[dev] = nullptr;
                c->err = std::string("hz_residual_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
                return HZ_ECUDA;
            }
        }
        scratch = g_na_ptr[dev];
    }
    k_na_resid<<<dim3(NA_CHUNKS, B), 256, 0, c->st>>>((const double2 *)u, (const double2 *)f, c->d_m, c->d_ax,
                                                      c->d_axh, c->d_az, c->d_azh, c->NX, c->NZ, c->h, c->omega,
                                                      scratch);
    k_na_final<<<(B + 127) / 128, 128, 0, c->st>>>(scratch, B, res);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        c->err = std::string("hz_residual_noalloc: launch failed: ") + cudaGetErrorString(e);
        return HZ_ECUDA;
    }
    return HZ_OK;
}
