// Solver context: problem description, decomposition descriptors, device
// operators and workspaces.  Internal to the library.
#pragma once
#include <map>
#include <memory>
#include <tuple>
#include <vector>

#include "../../include/hz.h"
#include "hz_common.cuh"

namespace hz {

// Online operators in one precision (T2 = double2 or float2).
template <class T2> struct Ops {
    T2 *cellW = nullptr;  // per cell: nz blocks of nx*nx (inverted Schur complements)
    T2 *cz = nullptr;     // per cell: z couplings (nz x nx, last row unused)
    T2 *F = nullptr, *E = nullptr, *S = nullptr;
    T2 *W = nullptr, *P = nullptr, *V = nullptr;  // inner block LU: W_j, P_j = W_j(:,0:nz) Z_j, V_j
    // compressed-block LU (opts.compress > 0): P_j ~ QP_j BP_j, V_j ~ QV_j BV_j (rank r);
    // STW_j = [BP_{j+1} W_j; BV_{j-1} W_j] (2r x 2nz), UX_j = [QP_j QV_j] (2nz x 2r),
    // MRN_j = [BP_j QP_{j-1}, BV_j QP_{j+1}, BV_j QV_{j+1}] (three r x r)
    T2 *STW = nullptr, *UX = nullptr, *MRN = nullptr;
    // the r-vector recursion of a layer as one matrix: ts = LAM ac (ac, ts in their
    // [C-1][2r] layout), applied as one product where a single layer is solved
    T2 *LAM = nullptr;
    // the sweep-step composites of each cell (offsets in CellDesc)
    T2 *CP2 = nullptr, *CP3 = nullptr, *CP1 = nullptr;
};

// Problem lists of batched GEMMs, kept on the device (built once per workspace).
template <class T2> struct ProbList {
    GemmProb<T2> *d = nullptr;
    int n = 0, max_tiles = 0;
    int kmax = 0;                 // longest K (both passes) of a problem
    int max_tiles32 = 0;          // most 32 x 32 tiles of a problem (small lists take that tile)
    int tc_max_tiles = 0;         // tensor-core GEMM: most 128 x 64 tiles of a problem,
    int tc_kchunks = 0;           // most K chunks of 16 (both passes), and
    long long tc_tiles = 0;       // tiles of the whole list
    long long tiles32 = 0;        // 32-row tiles of the whole list
    int max_m = 0, max_n = 0;     // most rows and most right-hand-side columns of a problem
    double bytes = 0, flops = 0;  // algorithmic traffic and real flops of one launch
};

// Workspace for one batch width B, in the working precision T2.
template <class T2> struct Work {
    int B = 0;
    T2 *vol = nullptr;     // cell volumes [tot_vol][B]: Newton potentials
    T2 *vol2 = nullptr;    // cell volumes for the reconstruction solve
    T2 *inner = nullptr;   // inner vectors [tot_inner][B]
    T2 *inner2 = nullptr;  // inner vectors [tot_inner][2B] (polarized operator, two input sets)
    T2 *inner_f = nullptr; // inner right-hand side of the Newton potentials (saved)
    T2 *innerH = nullptr;  // h_j = W_j g_j, B wide
    T2 *innerH2 = nullptr; // h_j = W_j g_j, 2B wide
                           // (compressed-block LU: innerH / innerH2 hold the right-hand sides g_j
                           // and inner / inner2 receive h_j, then x_j)
    T2 *ac = nullptr, *ts = nullptr;    // compressed-block LU recursion inputs / outputs [tot_ac][B]
    T2 *ac2 = nullptr, *ts2 = nullptr;  // the same, 2B wide
    T2 *lin = nullptr;     // layer-application inputs  [L][4][T][2B]
    T2 *lout = nullptr;    // layer-application outputs [L][4][T][2B]
    T2 *pa = nullptr, *pb = nullptr, *pc = nullptr;  // polarized vectors [K][4][T][B]
    T2 *Z = nullptr;       // FGMRES preconditioned basis [m][n_tr][B]
    // FP64 buffers
    double2 *V = nullptr;      // Arnoldi basis [m+1][n_tr][B]
    double2 *w64 = nullptr;    // [n_tr][B]
    double2 *rhs64 = nullptr;  // [n_tr][B]
    double2 *x64 = nullptr;    // [n_tr][B]
    double *dots = nullptr;    // reduction scratch
    double *hbuf = nullptr;    // [m+2][B] complex as 2 doubles
    double *hhost = nullptr;   // pinned mirror
    double2 *gsrc = nullptr;   // symmetric-form source / residual [NZ*NX][B]
    double2 *u = nullptr;      // FP64 solution [NZ*NX][B]
    double2 *io = nullptr;     // batch-outer staging [B][NZ*NX]
    const double2 *cur_src = nullptr;  // source of the current pass (nested inner level: reconstruction)
    double *rnorm = nullptr;   // [B] norms
    double *rhost = nullptr;   // pinned [4B]
    int restart = 0;
    // precomputed problem lists
    ProbList<T2> f_full, es_bot_A, es_top_B;  // apply_M (all layers)
    std::vector<ProbList<T2>> f_down, es_down; // per sweep step
    std::vector<ProbList<T2>> f_up, es_up;
    ProbList<T2> f_refl, es_refl;               // reflections (all layers)
    ProbList<T2> f_rec, e_newton;              // reconstruction F-step, Newton E-step
    std::vector<ProbList<T2>> f_layer, es_layer; // single-layer (component API)
    // h_j = W_j g_j problems ordered by layer; layers [l0, l1) are problems [hoff[l0], hoff[l1])
    ProbList<T2> hB, h2B;
    std::vector<int> hoff;
    // compressed-block LU: x_j += UX_j ts_j, layers [l0, l1) are problems [uoff[l0], uoff[l1]);
    // hB / h2B then also hold ac_j = STW_j g_j (layer by layer with the h_j problems)
    ProbList<T2> uxB, ux2B;
    std::vector<int> uoff;
    // compressed-block LU of one layer at a time: ts = LAM ac, problem l of layer l
    ProbList<T2> lamB, lam2B;
    // compressed-block LU sweep steps through the composites: [out += P2 in, ac = P1 in]
    // then (after ts = LAM ac) out += P3 ts, per step of the downward / upward sweeps
    std::vector<ProbList<T2>> cA_down, cC_down, cA_up, cC_up;
    ProbList<T2> cA_refl, cC_refl;  // the reflections (all layers) through the composites
    ProbList<T2> cA_M, cC_M;        // the polarized operator (both input sets) through the composites
    // persistent sweeps (FP32, <= 16 even columns): the phases of the downward and upward
    // sweeps, their algorithmic bytes / flops, and the grid barrier counter
    NwPhase *sw_down = nullptr, *sw_up = nullptr;
    int nsw_down = 0, nsw_up = 0;
    double sw_bytes[2] = {0, 0}, sw_flops[2] = {0, 0};
    unsigned *sw_bar = nullptr;
    std::vector<double> hbytes, hflops;  // per layer (B wide)
    std::vector<long long> htiles, utiles;  // 32-row tiles per layer of the h_j and x_j lists
};

}  // namespace hz

struct hz_ctx;
namespace hz {
// tensor-core GEMM (hz_tcgemm.cu): the split copy of operator block A (M x K,
// leading dimension lda), built on first use
const float *tc_split_operator(hz_ctx *c, const float2 *A, long long lda, int M, int K);
void tc_refresh_operators(hz_ctx *c);  // rebuild every split copy from the current operators
long long atc_floats(int M, int K);
}  // namespace hz

struct hz_ctx {
    // problem
    int n_x = 0, n_z = 0, p = 0, L = 0, C = 0;
    double omega = 0, h = 0, pml_C = 0;
    int NX = 0, NZ = 0;
    hz_opts opts{};
    std::vector<int> rows, cols;
    cudaStream_t st = nullptr;
    std::string err;
    bool factored = false;
    int nl = 0;  // kernel launches counter for the current call
    // decomposition
    std::vector<hz::CellDesc> cells;
    std::vector<hz::LayerDesc> layers;
    hz::CellDesc *d_cells = nullptr;
    hz::LayerDesc *d_layers = nullptr;
    int *d_layer_ids = nullptr;  // 0..L-1
    long long tot_vol = 0, tot_W = 0, tot_F = 0, tot_E = 0, tot_S = 0, tot_K = 0;
    long long tot_inner = 0, tot_Wi = 0, tot_P = 0, tot_V = 0;
    int lr_r = 0;  // compressed-block LU rank (0: dense inner factors)
    long long tot_lr = 0, tot_m = 0, tot_ac = 0, tot_lam = 0, tot_cp2 = 0, tot_cp3 = 0, tot_cp1 = 0;
    int max_nx = 0, max_nz = 0, max_no = 0;
    // global medium and PML profiles (FP64)
    std::vector<double> h_m;  // host copy of the medium (local model updates compare against it)
    double *d_m = nullptr;
    double2 *d_ax = nullptr, *d_axh = nullptr, *d_az = nullptr, *d_azh = nullptr;
    // row-scaled global operator: diagonal, +x and +z couplings, and alpha_x alpha_z (FP64)
    double2 *d_gdiag = nullptr, *d_gcx = nullptr, *d_gcz = nullptr, *d_gD = nullptr;
    double2 *d_ginvD = nullptr;  // 1 / (alpha_x alpha_z)
    double2 *d_ggam = nullptr;   // -1 / (alpha_x h^2) per global column (z coupling at interface rows)
    double2 *d_lbeta = nullptr;  // -1 / (alpha_z h^2) per layer row, layer-local PML (x coupling at cell interfaces)
    long long tot_z = 0;
    hz::CellDesc *d_gcell = nullptr;
    // operators
    hz::Ops<double2> o64;
    hz::Ops<float2> o32;
    std::unique_ptr<hz::Work<double2>> w64;
    std::unique_ptr<hz::Work<float2>> w32;
    // kernel timing (opts.time_kernels): event pairs per hot-kernel class
    struct KT {
        int cls;
        cudaEvent_t a, b;
        double bytes, flops;
    };
    std::vector<KT> kt_open;
    std::vector<cudaEvent_t> ev_pool;
    int kt_launches[3] = {0, 0, 0};
    double kt_ms[3] = {0, 0, 0}, kt_bytes[3] = {0, 0, 0}, kt_flops[3] = {0, 0, 0};
    cudaEvent_t ev_get();
    void kt_begin(int cls, double bytes, double flops);
    void kt_end();
    void kt_collect();  // synchronises; folds open event pairs into kt_*
    void kt_reset();
    // host<->device staging of user arrays
    double2 *stage = nullptr;
    long long stage_n = 0;
    int *d_flag = nullptr;
    int *d_err = nullptr;  // device status block (error word + wait limit, see hz_common.cuh)
    // host-side fault injection (environment HZ_FAULT, read at hz_setup): the
    // failure paths of the library are exercised without faulting a GPU
    enum { FAULT_NONE = 0, FAULT_ALLOC, FAULT_NAN, FAULT_NOCONV, FAULT_SINGULAR };
    int fault = FAULT_NONE;
    long long fault_n = 1;    // FAULT_ALLOC: the n-th device allocation after hz_setup fails
    long long n_dalloc = 0;   // device allocations made so far
    int dev = 0;           // CUDA device current at hz_setup
    void *gemm_ws = nullptr;  // split-K partial tiles of the batched GEMM (sized for double2)
    float *wtc = nullptr;     // split TF32 W blocks of the tensor-core cell solve (null: SIMT cell solve)
    int *gemm_cnt = nullptr;  // split-K arrival counters (zero between launches)
    float2 *tcg_ws = nullptr; // split-K partial tiles of the tensor-core GEMM (GEMM_TC_WS_TILES)
    int *tcg_cnt = nullptr;   // its arrival counters
    float2 *nw_ws = nullptr;  // split-K partial tiles of the narrow GEMM (NW_WS_SLOTS)
    int *nw_cnt = nullptr;    // its arrival counters
    // TF32 split copies of the operator blocks the tensor-core GEMM reads, keyed by
    // (block address, leading dimension, rows, columns), in device slabs
    std::map<std::tuple<const void *, long long, int, int>, float *> tca;
    std::vector<void *> tca_slabs;
    size_t tca_used = 0, tca_cap = 0;
    bool tca_pending = false;  // split copies enqueued since the last stream synchronisation
    // right-hand-side lanes (opts.rhs_lanes): contexts that share this one's
    // decomposition, operators and split copies but own a stream, workspaces,
    // error word and timers
    std::vector<hz_ctx *> lanes;
    hz_ctx *parent = nullptr;  // set on a lane
    int group_n = 1;           // contexts of the solve in progress (persistent sweeps need the GPU alone)
    // inner nested polarized traces (opts.inner = HZ_INNER_NESTED): per layer, a
    // context of the layer's box with x and z swapped (its layers are the cells),
    // a lane of it for 2B-wide applications, and FP64 source / solution volumes
    // on its grid ([2B][NX][nz_l]); inner GMRES iterations of the current call
    std::vector<hz_ctx *> inner_ctx, inner_wide;
    std::vector<double2 *> nsrc, nsol;
    int n_bw = 0;
    long long inner_its = 0;
    bool nested() const { return opts.inner == HZ_INNER_NESTED; }
    bool own_stream = false;
    // allocations
    std::map<void *, size_t> allocs;
    long long dev_bytes = 0;

    void *dalloc(size_t bytes);
    void dfree(void *p);
    bool mixed() const { return opts.precision == HZ_MIXED; }
    long long n_tr() const { return 4LL * (L - 1) * NX; }
};

namespace hz {
void build_decomposition(hz_ctx *c);
void factor_all(hz_ctx *c);
void factor_layers(hz_ctx *c, const std::vector<int> &lays, bool first);
void init_global_alpha(hz_ctx *c);
template <class T2> int solve_impl(hz_ctx *c, const double2 *f_dev, int B, double2 *u_dev, hz_stats *st, bool scale_src);
template <class T2>
int solve_group_impl(const std::vector<hz_ctx *> &cs, const std::vector<const double2 *> &f_dev, int B,
                     const std::vector<double2 *> &u_dev, std::vector<hz_stats> &stats, bool scale_src);
template <class T2> void comp_cell_solve(hz_ctx *c, int ci, const double2 *g_dev, int B, double2 *x_dev);
template <class T2> void comp_layer_green(hz_ctx *c, int l, const double2 *tr_dev, int mask, int B, double2 *out_dev);
template <class T2> void comp_polar(hz_ctx *c, int which, const double2 *x_dev, int B, double2 *y_dev);
template <class T2> void comp_residual(hz_ctx *c, const double2 *u_dev, const double2 *f_dev, int B, double *res_host);
void comp_traces(hz_ctx *c, const double2 *u_dev, int B, double2 *tr_dev);
template <class T2> void comp_reconstruct(hz_ctx *c, const double2 *f_dev, const double2 *tr_dev, int B, double2 *u_dev);
template <class T2> Ops<T2> &ops(hz_ctx *c);
template <class T2> Work<T2> &work(hz_ctx *c, int B);
hz_ctx *make_lane(hz_ctx *c);
}  // namespace hz
