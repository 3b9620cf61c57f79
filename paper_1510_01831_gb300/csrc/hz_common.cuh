// Shared types and device helpers of the CUDA path (complex arithmetic,
// problem descriptors, kernel declarations).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/hz.h"

namespace hz {

// ------------------------------------------------------ status block ---
// Device status block of a context (16 bytes, 8-byte aligned): int 0 is the
// error word (1 = a bounded wait in a kernel gave up), bytes 8-15 hold the
// limit of every bounded wait in nanoseconds (hz_opts.wait_ms).  Kernels
// receive the block as `int *err`.
__device__ __forceinline__ unsigned long long wait_limit_ns(const int *err) {
    return *reinterpret_cast<const volatile unsigned long long *>(err + 2);
}
// limit after a thread has given up once (draining its own copies)
constexpr unsigned long long DRAIN_WAIT_NS = 1000000ull;

// ------------------------------------------------------------ complex ---
template <class T> struct cx;
template <> struct cx<double> { using t = double2; };
template <> struct cx<float> { using t = float2; };

__host__ __device__ inline double2 mk(double a, double b) { return make_double2(a, b); }
__host__ __device__ inline float2 mk(float a, float b) { return make_float2(a, b); }

__host__ __device__ inline double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline double2 operator*(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline double2 operator*(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__host__ __device__ inline float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline float2 operator*(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline float2 operator*(float s, float2 a) { return make_float2(s * a.x, s * a.y); }

// acc += a * b with fused multiply-adds
__device__ __forceinline__ void cmac(double2 &acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cmac(float2 &acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}
__host__ __device__ inline double2 cdiv(double2 a, double2 b) {
    // Smith's algorithm for a / b
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, d = b.x + b.y * r;
        return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
    } else {
        double r = b.x / b.y, d = b.x * r + b.y;
        return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
    }
}
__host__ __device__ inline double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }

template <class T2> __device__ __forceinline__ T2 czero();
template <> __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }

__device__ __forceinline__ double2 to2(double2 a, double2) { return a; }
__device__ __forceinline__ float2 to2(double2 a, float2) { return make_float2((float)a.x, (float)a.y); }
__device__ __forceinline__ double2 to2(float2 a, double2) { return make_double2(a.x, a.y); }
__device__ __forceinline__ float2 to2(float2 a, float2) { return a; }

// ------------------------------------------------------- descriptors ---
// One cell (l, c) of the nested decomposition.  Local arrays are row-major
// [nz][nx] with nz = n + 2p rows and nx = w + 2p columns; local array column
// jx maps to global array column t + jx, local row jz to global row s + jz.
struct CellDesc {
    int l, c;
    int top, bot, left, right;  // neighbour flags: layer above/below, cell left/right
    int nx, nz;          // extended cell size
    int w, n;            // interior columns / rows
    int t, s;            // global interior column / row offsets (t_c, s_l)
    int own_lo, no;      // owned local columns [own_lo, own_lo + no)
    int row_lo, row_hi;  // owned local rows [row_lo, row_hi) of the layer
    long long vol_off;   // cell volume buffer offset (in grid points; x B for RHS-major)
    long long w_off;     // block-tridiagonal inverse blocks: nz blocks of nx rows x ldw (row stride)
    int ldw;             // row stride of the W blocks: nx rounded up to even (16-byte rows for async copies)
    long long cz_off;    // z-couplings between consecutive rows: (nz-1) x nx
    long long F_off;     // F: (2 nz) x (4 no)
    long long E_off;     // E: (4 no) x (4 nz)
    long long S_off;     // S: (4 no) x (4 no)
    long long K_off;     // K (offline only): (2 nz) x (4 nz)
    long long tc_off;    // split TF32 copy of the W blocks for the tensor-core cell solve (floats)
    // compressed-block LU only: the sweep step of the layer as three products whose
    // operators are composed offline.  The inputs of cell c's composite are the owned
    // columns of cells c-1, c, c+1 (a contiguous range of Lt columns of each trace row,
    // cell c's own at offset cl); P2 (4 no x 4 Lt) = E W F + S, P3 (4 no x 4r) = E UX on
    // [ts of interface c-1; ts of interface c]; P1 (2r x 4 (no + no of cell c+1)) =
    // STW F of interface c (cells c, c+1; none for the last cell)
    long long P2_off, P3_off, P1_off;
    int cl, Lt;
};

// One layer: its inner SIE over the C-1 cell interfaces.
struct LayerDesc {
    int n, nz, s, C;
    int row_lo, row_hi;
    int cell0;           // index of its first cell
    long long inner_off; // inner vector offset: (C+1) slots of 2 nz (slot 0 and C are zero pads)
    long long W_off;     // C-1 blocks (2nz)^2
    long long P_off;     // C-1 blocks (2nz)^2: P_j = W_j(:, 0:nz) Z_j (slot 0 unused)
    long long V_off;     // C-1 blocks (2nz)^2 (last unused)
    long long zoff;      // offset of the layer's per-row arrays (nz entries)
    // compressed-block LU (rank r of the context): C-1 blocks of 2r x 2nz (STW, and
    // their transposes' shape 2nz x 2r for UX), C-1 triples of r x r (MRN), C-1 vectors
    // of 2r per right-hand side (the recursion's inputs AC and outputs TS), and the
    // recursion as one linear map TS = LAM AC (2r(C-1) x 2r(C-1))
    long long lr_off, m_off, ac_off, lam_off;
};

// Batched, segmented complex GEMM problem:  Y (+)= alpha (A X + A2 X2)
//   A : M x K row-major (lda); A2 : M x K2 (lda2), optional (K2 = 0)
//   X row k lives at X[k / xseg] + (k % xseg) * ldx (N contiguous entries)
//   Y row m lives at Y[m / yseg] + (m % yseg) * ldy
template <class T2> struct GemmProb {
    const T2 *A;
    long long lda;
    int M, K, N;
    int xseg, yseg;
    long long ldx, ldy;
    const T2 *X[4];
    T2 *Y[4];
    int beta;     // 0 overwrite, 1 accumulate
    float alpha;  // real scale
    const T2 *A2;
    long long lda2;
    int K2, xseg2;
    long long ldx2;
    const T2 *X2[4];
    // tensor-core GEMM only: TF32 split copies of A and A2 (per 128-row tile and
    // 16-column chunk, canonical MMA layout; null elsewhere)
    const float *Atc, *A2tc;
};

// ------------------------------------------------------------ errors ---
struct Err {
    int code = 0;
    std::string msg;
};

#define HZ_CU(call)                                                                  \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            throw hz::CudaError(e_, #call, __FILE__, __LINE__);                      \
        }                                                                            \
    } while (0)

struct CudaError {
    cudaError_t e;
    std::string what;
    CudaError(cudaError_t e_, const char *call, const char *file, int line) : e(e_) {
        char b[512];
        snprintf(b, sizeof b, "%s failed: %s (%s:%d)", call, cudaGetErrorString(e_), file, line);
        what = b;
    }
};
struct HzError {
    int code;
    std::string what;
    HzError(int c, const std::string &w) : code(c), what(w) {}
};

// ------------------------------------------------- kernel launchers ---
// (defined in hz_kernels.cu; all launch on `st` and count launches in *nl)
// cfg: output tile of a CTA, 0 = 64 x 32 (GBM x GBN), 1 = 32 x 32, 2 = 64 x 16;
// max_tiles counts tiles of that shape (gemm_tiles)
template <class T2>
void launch_gemm(const GemmProb<T2> *d_probs, int nprob, int max_tiles, int split, T2 *ws, int *cnt, cudaStream_t st,
                 int *nl, int cfg = 0);
int gemm_tiles(int M, int N, int cfg);
// skinny batched GEMM: every problem's N <= nmax <= 16; max_m = most rows of a problem
template <class T2>
void launch_gemm_skinny(const GemmProb<T2> *d_probs, int nprob, int max_m, int nmax, cudaStream_t st, int *nl);
// narrow batched GEMM: K block, warps per CTA, columns, CTAs resident per SM, and the
// split-K workspace (partial 32 x NW_NB tiles and their counters)
constexpr int NW_KB = 16, NW_WPC = 4, NW_NB = 16, NW_CTAS_PER_SM = 4, NW_WS_SLOTS = 2048;
// narrow batched GEMM (FP32): every problem's N <= nmax <= NW_NB; max_tiles = most 32-row
// tiles of a problem; split = K slices per tile (<= 8; > 1 needs ws and cnt, whose
// slots are problem * max_tiles + tile)
void launch_gemm_narrow(const GemmProb<float2> *d_probs, int nprob, int max_tiles, int nmax, int split, float2 *ws,
                        int *cnt, cudaStream_t st, int *nl);
// persistent narrow sweep: phases run in order, each a list of n problems (<= NW_NB
// columns, N and ldx even, 16-byte aligned right-hand-side rows) with max_tiles 32-row
// tiles and split K slices; grid <= narrow_sweep_grid() CTAs (all co-resident), bar a
// device counter, err the context's status block
struct NwPhase {
    const GemmProb<float2> *d;
    int n, max_tiles, split;
};
int narrow_sweep_grid();
void launch_narrow_sweep(const NwPhase *d_ph, int nph, float2 *ws, int *cnt, unsigned *bar, int *err, int grid,
                         cudaStream_t st, int *nl);
// batched GEMM tile (complex outputs) and K step
constexpr int GBM = 64, GBN = 32, GBK = 16;
// split-K is used while a launch has fewer tiles than this; its workspace
// holds at most 2x this many partial tiles
constexpr int GEMM_SPLIT_TILES = 304;

// tensor-core batched GEMM (mixed precision): 128 x 64 output tiles, K chunks of
// 16; split-K while a launch has fewer tiles than GEMM_TC_SPLIT_TILES, with a
// workspace of at most GEMM_TC_WS_TILES partial tiles (defined in hz_tcgemm.cu)
constexpr int GT_M = 128, GT_N = 64, GT_KC = 16;
constexpr int GEMM_TC_SPLIT_TILES = 152, GEMM_TC_WS_TILES = 1024;
// launches with fewer (tiles x K chunks) than this take the SIMT kernel
constexpr long long GEMM_TC_MIN_WORK = 600;
void launch_gemm_tc(const GemmProb<float2> *d_probs, int nprob, int max_tiles, int split, float2 *ws, int *cnt,
                    int *err, cudaStream_t st, int *nl);

// tensor-core cell solve (mixed precision, cells up to 128 columns)
size_t cell_chain_tc_smem(int max_nx);
long long cell_tc_floats(int nx, int nz);
void build_wtc(const CellDesc *d_cells, int ncell, const double2 *W, float *wtc, cudaStream_t st, int *nl);
void launch_wait_check(int *err, cudaStream_t st, int *nl);
void launch_cell_chain_tc(const CellDesc *d_cells, int ncell, const float *wtc, const float2 *cz, float2 *vol, int B,
                          int max_nx, int *err, cudaStream_t st, int *nl);
template <class T2>
void launch_cell_chain(const CellDesc *d_cells, int ncell, const T2 *W, const T2 *cz, T2 *vol, int B,
                       int max_nx, cudaStream_t st, int *nl);

template <class T2>
void launch_inner_sweep(const LayerDesc *d_layers, const int *d_layer_ids, int nlayer, const T2 *P, const T2 *V,
                        const T2 *H, T2 *X, int B, int max_n2, int *err, cudaStream_t st, int *nl,
                        bool tune = false);

// offline (FP64)
void launch_cell_coeffs(const CellDesc *d_cells, int ncell, const double *m, int NX, double omega, double h,
                        double C, int p, double2 *diag, double2 *cx, double2 *cz, cudaStream_t st, int *nl);
void launch_cell_factor(const CellDesc *d_cells, int ncell, const double2 *diag, const double2 *cx,
                        const double2 *cz, double2 *W, int max_nx, int *d_info, cudaStream_t st, int *nl);
void launch_gj_inverse(double2 *const *d_mats, const int *d_n, int nmat, int max_n, int *d_info,
                       cudaStream_t st, int *nl);

}  // namespace hz
