// Generic kernels of the CUDA path:
//   * batched segmented complex GEMM (F, E, S steps of eq. (factorization))
//   * block-tridiagonal chain solves with explicitly inverted Schur blocks:
//     cell volume solves (local solves of Alg. inner_solver) and the inner
//     compressed-block LU sweeps of Section 4.2.2
//   * pivoted Gauss-Jordan inversion (offline, FP64)
#include <cooperative_groups.h>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>

#include "hz_common.cuh"

namespace hz {

// ================================================================ GEMM ===


// asynchronous copy of one complex element (8 or 16 bytes) into shared memory;
// bytes = 0 fills it with zeros
template <int SZ> __device__ __forceinline__ void gemm_cp(void *dst, const void *src, unsigned bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(d), "l"(src), "n"(SZ), "r"(bytes) : "memory");
}
// 16-byte asynchronous copy that bypasses L1 (data written by other CTAs of the same launch)
__device__ __forceinline__ void gemm_cp16cg(void *dst, const void *src, unsigned bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void gemm_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void gemm_cp_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
// FP32: two stages filled through registers (measured faster here); FP64: a 3-stage ring of asynchronous copies
template <class T2> constexpr int gemm_stages() { return sizeof(T2) == 8 ? 2 : 3; }

// BM x BN complex outputs per CTA of 256 threads (16 x 16): (BM / 16) x (BN / 16)
// per thread, K steps of GBK.  FP32: the next step's operands are loaded into
// registers during the current step's products and stored to the other of two
// shared-memory buffers.  FP64: the K steps of both operand pairs, laid end to
// end, flow through a 3-stage ring filled by asynchronous copies two steps ahead.
template <class T2, int BM, int BN>
__global__ void __launch_bounds__(256) k_gemm(const GemmProb<T2> *__restrict__ probs, int S, T2 *ws, int *cnt,
                                              int max_tiles) {
    constexpr int MI = BM / 16, NJ = BN / 16, NST = gemm_stages<T2>();
    __shared__ GemmProb<T2> P;
    extern __shared__ __align__(16) unsigned char gsm[];
    T2 (*As)[GBK][BM + 1] = reinterpret_cast<T2 (*)[GBK][BM + 1]>(gsm);
    T2 (*Xs)[GBK][BN] = reinterpret_cast<T2 (*)[GBK][BN]>(gsm + sizeof(T2) * NST * GBK * (BM + 1));
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    if (tid == 0) P = probs[blockIdx.y];
    __syncthreads();
    const int M = P.M, N = P.N;
    const int tilesM = (M + BM - 1) / BM, tilesN = (N + BN - 1) / BN;
    const int tile = blockIdx.x / S, sp = blockIdx.x % S;
    if (tile >= tilesM * tilesN) return;
    // split sp of S takes a GBK-aligned slice of the K range of both passes laid end to end
    const int K1 = max(P.K, 0), Kt = K1 + max(P.K2, 0);
    const int per = ((Kt + S - 1) / S + GBK - 1) / GBK * GBK;
    const int kb = min(Kt, sp * per), ke = min(Kt, kb + per);
    const int m0 = (tile % tilesM) * BM, n0 = (tile / tilesM) * BN;
    // this split's part of each pass, in the pass's own K coordinates, and its steps
    const int klo0 = min(kb, K1), kend0 = min(ke, K1);
    const int klo1 = max(kb - K1, 0), kend1 = max(ke - K1, 0);
    const int ns0 = kend0 > klo0 ? (kend0 - klo0 + GBK - 1) / GBK : 0;
    const int ns1 = kend1 > klo1 ? (kend1 - klo1 + GBK - 1) / GBK : 0;
    const int nk = ns0 + ns1;
    T2 acc[MI][NJ];
#pragma unroll
    for (int i = 0; i < MI; i++)
#pragma unroll
        for (int j = 0; j < NJ; j++) acc[i][j] = czero<T2>();
    // copy slots of this thread: A elements (mm, kk) for q < AQ, X elements (kk, nn) for q < XQ
    constexpr int AR = 256 / GBK, AQ = BM / AR;  // A rows per pass, passes
    constexpr int XR = 256 / BN, XQ = GBK / XR;  // X rows per pass, passes
    const int a_kk = tid % GBK, a_mm = tid / GBK;  // + AR q rows
    const int x_nn = tid % BN, x_kk = tid / BN;   // + XR q rows
    if constexpr (sizeof(T2) == 8) {
        T2 ra[AQ], rx[XQ];
        int buf = 0;
        for (int pass = 0; pass < 2; pass++) {
            const T2 *A = pass ? P.A2 : P.A;
            const long long lda = pass ? P.lda2 : P.lda;
            const int xseg = pass ? P.xseg2 : P.xseg;
            const long long ldx = pass ? P.ldx2 : P.ldx;
            const T2 *const *Xp = pass ? P.X2 : P.X;
            // this split's part of the pass, in the pass's own K coordinates
            const int off = pass ? K1 : 0, Kp = pass ? Kt - K1 : K1;
            const int klo = max(kb - off, 0), K = min(ke - off, Kp);
            if (K <= klo) continue;
            auto load = [&](int k0) {
#pragma unroll
                for (int q = 0; q < AQ; q++) {
                    const int gm = m0 + a_mm + AR * q, gk = k0 + a_kk;
                    ra[q] = (gm < M && gk < K) ? A[(long long)gm * lda + gk] : czero<T2>();
                }
#pragma unroll
                for (int q = 0; q < XQ; q++) {
                    const int gk = k0 + x_kk + XR * q, gn = n0 + x_nn;
                    T2 v = czero<T2>();
                    if (gk < K && gn < N) {
                        const int sg = gk / xseg;
                        v = Xp[sg][(long long)(gk - sg * xseg) * ldx + gn];
                    }
                    rx[q] = v;
                }
            };
            load(klo);
            for (int k0 = klo; k0 < K; k0 += GBK) {
#pragma unroll
                for (int q = 0; q < AQ; q++) As[buf][a_kk][a_mm + AR * q] = ra[q];
#pragma unroll
                for (int q = 0; q < XQ; q++) Xs[buf][x_kk + XR * q][x_nn] = rx[q];
                __syncthreads();
                if (k0 + GBK < K) load(k0 + GBK);  // in flight during the products below
#pragma unroll
                for (int kk = 0; kk < GBK; kk++) {
                    T2 a[MI], x[NJ];
#pragma unroll
                    for (int i = 0; i < MI; i++) a[i] = As[buf][kk][ty + 16 * i];
#pragma unroll
                    for (int j = 0; j < NJ; j++) x[j] = Xs[buf][kk][tx + 16 * j];
#pragma unroll
                    for (int i = 0; i < MI; i++)
#pragma unroll
                        for (int j = 0; j < NJ; j++) cmac(acc[i][j], a[i], x[j]);
                }
                buf ^= 1;  // the other buffer is free: every thread passed this chunk's barrier
            }
        }
    } else {
        auto issue = [&](int t) {  // copies of step t into stage t % NST
            const int bf = t % NST;
            const bool p2 = t >= ns0;
            const int k0 = p2 ? klo1 + (t - ns0) * GBK : klo0 + t * GBK, K = p2 ? kend1 : kend0;
            const T2 *A = p2 ? P.A2 : P.A;
            const long long lda = p2 ? P.lda2 : P.lda;
            const int xseg = p2 ? P.xseg2 : P.xseg;
            const long long ldx = p2 ? P.ldx2 : P.ldx;
            const T2 *const *Xp = p2 ? P.X2 : P.X;
#pragma unroll
            for (int q = 0; q < AQ; q++) {
                const int gm = m0 + a_mm + AR * q, gk = k0 + a_kk;
                const bool ok = gm < M && gk < K;
                gemm_cp<sizeof(T2)>(&As[bf][a_kk][a_mm + AR * q], ok ? A + (long long)gm * lda + gk : A,
                                    ok ? (unsigned)sizeof(T2) : 0u);
            }
#pragma unroll
            for (int q = 0; q < XQ; q++) {
                const int gk = k0 + x_kk + XR * q, gn = n0 + x_nn;
                const bool ok = gk < K && gn < N;
                const T2 *src = Xp[0];
                if (ok) {
                    const int sg = gk / xseg;
                    src = Xp[sg] + (long long)(gk - sg * xseg) * ldx + gn;
                }
                gemm_cp<sizeof(T2)>(&Xs[bf][x_kk + XR * q][x_nn], src, ok ? (unsigned)sizeof(T2) : 0u);
            }
        };
#pragma unroll
        for (int t = 0; t < NST - 1; t++) {  // prologue: the first NST - 1 steps in flight
            if (t < nk) issue(t);
            gemm_cp_commit();
        }
        for (int t = 0; t < nk; t++) {
            gemm_cp_wait<NST - 2>();  // this thread's copies of step t have landed
            __syncthreads();          // everyone's have; and every thread is done with step t - 1
            if (t + NST - 1 < nk) issue(t + NST - 1);  // into the stage of step t - 1
            gemm_cp_commit();
            const int bf = t % NST;
#pragma unroll
            for (int kk = 0; kk < GBK; kk++) {
                T2 a[MI], x[NJ];
#pragma unroll
                for (int i = 0; i < MI; i++) a[i] = As[bf][kk][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < NJ; j++) x[j] = Xs[bf][kk][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < MI; i++)
#pragma unroll
                    for (int j = 0; j < NJ; j++) cmac(acc[i][j], a[i], x[j]);
            }
        }
        gemm_cp_wait<0>();
    }
    const float al = P.alpha;
    if (S > 1) {
        // split-K: every split stores its partial tile; the last split of the
        // tile to finish adds the partials in split order (deterministic) and
        // writes the output, then re-arms the tile's counter
        const long long slot = (long long)blockIdx.y * max_tiles + tile;
        T2 *mine = ws + (slot * S + sp) * (BM * BN);
#pragma unroll
        for (int i = 0; i < MI; i++)
#pragma unroll
            for (int j = 0; j < NJ; j++) mine[(ty + 16 * i) * BN + tx + 16 * j] = acc[i][j];
        __threadfence();
        __syncthreads();
        __shared__ int last;
        if (tid == 0) last = atomicAdd(&cnt[slot], 1) == S - 1;
        __syncthreads();
        if (!last) return;
        __threadfence();
#pragma unroll
        for (int i = 0; i < MI; i++)
#pragma unroll
            for (int j = 0; j < NJ; j++) {
                T2 v = czero<T2>();
                for (int q = 0; q < S; q++) {
                    const T2 *pq = ws + (slot * S + q) * (BM * BN) + (ty + 16 * i) * BN + tx + 16 * j;
                    const T2 w = __ldcg(pq);
                    v.x += w.x;
                    v.y += w.y;
                }
                acc[i][j] = v;
            }
        if (tid == 0) cnt[slot] = 0;
    }
#pragma unroll
    for (int i = 0; i < MI; i++) {
        const int m = m0 + ty + 16 * i;
        if (m >= M) continue;
        const int sg = m / P.yseg;
        T2 *row = P.Y[sg] + (long long)(m - sg * P.yseg) * P.ldy;
#pragma unroll
        for (int j = 0; j < NJ; j++) {
            const int n = n0 + tx + 16 * j;
            if (n >= N) continue;
            T2 v = acc[i][j];
            v.x *= al;
            v.y *= al;
            row[n] = P.beta ? row[n] + v : v;
        }
    }
}

// two complex values held as one 16-byte (float) or two 16-byte (double) registers
template <class T2> struct Pair {
    T2 a, b;
};
template <class T2> __device__ __forceinline__ Pair<T2> ld_pair(const T2 *p) {
    return Pair<T2>{p[0], p[1]};
}
template <> __device__ __forceinline__ Pair<float2> ld_pair<float2>(const float2 *p) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    return Pair<float2>{make_float2(v.x, v.y), make_float2(v.z, v.w)};
}

// Skinny form of the batched GEMM for short lists whose right-hand-side panels
// have at most 16 columns (a sweep step's products for batches of <= 16
// sources): every operator element is read once and meets all N columns, and
// the K loop keeps the next block's loads in flight.  A CTA of 4 warps owns 32
// rows of one problem (lane = row); the K range of both operand pairs, laid end
// to end, is cut into four slices, one per warp.  Per block of 32 K a warp
// loads 32 x 32 of A (coalesced rows) and 32 x 16 of X into registers one block
// ahead, stores them to its shared-memory area, and reads A back transposed
// (its own row) and X as 16-byte broadcasts.  The four partial sums are added
// in warp order (deterministic) and written with alpha / beta.
constexpr int SK_NB = 16;
template <class T2>
__global__ void __launch_bounds__(128) k_gemm_skinny(const GemmProb<T2> *__restrict__ probs) {
    __shared__ GemmProb<T2> P;
    extern __shared__ __align__(16) unsigned char gsm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    T2 *Aw = reinterpret_cast<T2 *>(gsm) + warp * (32 * 33 + 32 * SK_NB);  // [32 rows][33]
    T2 *Xw = Aw + 32 * 33;                                                // [32 k][16]
    if (tid == 0) P = probs[blockIdx.y];
    __syncthreads();
    const int M = P.M, N = P.N;
    const int m0 = blockIdx.x * 32;
    if (m0 >= M) return;  // uniform over the CTA
    const int K1 = max(P.K, 0), Kt = K1 + max(P.K2, 0);
    const int per = ((Kt + 3) / 4 + 31) / 32 * 32;
    const int kb = min(Kt, warp * per), ke = min(Kt, kb + per);
    // this warp's part of each pass (pass coordinates) and its blocks of 32
    const int lo0 = min(kb, K1), hi0 = min(ke, K1), lo1 = max(kb - K1, 0), hi1 = max(ke - K1, 0);
    const int c0 = hi0 > lo0 ? (hi0 - lo0 + 31) / 32 : 0, c1 = hi1 > lo1 ? (hi1 - lo1 + 31) / 32 : 0;
    const int nblk = c0 + c1;
    // X element this lane loads for row i of a block: lanes 0-15 even rows, 16-31 odd rows
    const int xn = lane & 15, xr0 = lane >> 4;
    T2 ra[32], rx[16];
    auto load = [&](int t) {
        const bool p2 = t >= c0;
        const int k0 = p2 ? lo1 + 32 * (t - c0) : lo0 + 32 * t, hi = p2 ? hi1 : hi0;
        const T2 *A = p2 ? P.A2 : P.A;
        const long long lda = p2 ? P.lda2 : P.lda;
        const int xseg = p2 ? P.xseg2 : P.xseg;
        const long long ldx = p2 ? P.ldx2 : P.ldx;
        const T2 *const *Xp = p2 ? P.X2 : P.X;
        const bool kin = k0 + lane < hi;
#pragma unroll
        for (int i = 0; i < 32; i++) {
            const int gm = m0 + i;
            ra[i] = (gm < M && kin) ? A[(long long)gm * lda + k0 + lane] : czero<T2>();
        }
#pragma unroll
        for (int i = 0; i < 16; i++) {
            const int gk = k0 + 2 * i + xr0;
            T2 v = czero<T2>();
            if (gk < hi && xn < N) {
                const int sg = gk / xseg;
                v = Xp[sg][(long long)(gk - sg * xseg) * ldx + xn];
            }
            rx[i] = v;
        }
    };
    T2 acc[SK_NB];
#pragma unroll
    for (int n = 0; n < SK_NB; n++) acc[n] = czero<T2>();
    if (nblk > 0) load(0);
    for (int t = 0; t < nblk; t++) {
        __syncwarp();  // the previous block's reads of Aw / Xw are done
#pragma unroll
        for (int i = 0; i < 32; i++) Aw[i * 33 + lane] = ra[i];
#pragma unroll
        for (int i = 0; i < 16; i++) Xw[(2 * i + xr0) * SK_NB + xn] = rx[i];
        __syncwarp();
        if (t + 1 < nblk) load(t + 1);  // in flight during this block's products
        const bool p2 = t >= c0;
        const int k0 = p2 ? lo1 + 32 * (t - c0) : lo0 + 32 * t;
        const int kc = min(32, (p2 ? hi1 : hi0) - k0);
        for (int kk = 0; kk < kc; kk++) {
            const T2 a = Aw[lane * 33 + kk];
            const T2 *xr = Xw + kk * SK_NB;
#pragma unroll
            for (int n = 0; n < SK_NB; n += 2) {
                const Pair<T2> x = ld_pair(xr + n);
                cmac(acc[n], a, x.a);
                cmac(acc[n + 1], a, x.b);
            }
        }
    }
    __syncthreads();  // every warp is done with its blocks: the buffers hold the partial sums now
    T2 *red = reinterpret_cast<T2 *>(gsm);  // [4][32][16]
#pragma unroll
    for (int n = 0; n < SK_NB; n++) red[(warp * 32 + lane) * SK_NB + n] = acc[n];
    __syncthreads();
    const float al = P.alpha;
    for (int e = tid; e < 32 * N; e += 128) {
        const int r = e / N, n = e % N, m = m0 + r;
        if (m >= M) continue;
        T2 v = red[r * SK_NB + n];
#pragma unroll
        for (int w = 1; w < 4; w++) v = v + red[(w * 32 + r) * SK_NB + n];
        v.x *= al;
        v.y *= al;
        const int sg = m / P.yseg;
        T2 *row = P.Y[sg] + (long long)(m - sg * P.yseg) * P.ldy;
        row[n] = P.beta ? row[n] + v : v;
    }
}

template <class T2>
void launch_gemm_skinny(const GemmProb<T2> *d_probs, int nprob, int max_m, int nmax, cudaStream_t st, int *nl) {
    if (nprob <= 0 || max_m <= 0) return;
    if (nmax > SK_NB) throw HzError(HZ_EINVAL, "skinny GEMM: too many columns");
    dim3 grid((max_m + 31) / 32, nprob);
    const size_t sm = sizeof(T2) * 4 * (32 * 33 + 32 * SK_NB);
    static bool attr = false;
    if (!attr) {  // FP64 needs more than the default 48 KB
        HZ_CU(cudaFuncSetAttribute(k_gemm_skinny<T2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        attr = true;
    }
    k_gemm_skinny<T2><<<grid, 128, sm, st>>>(d_probs);
    HZ_CU(cudaGetLastError());
    if (nl) (*nl)++;
}
template void launch_gemm_skinny<float2>(const GemmProb<float2> *, int, int, int, cudaStream_t, int *);

// Narrow form of the batched GEMM (FP32) for panels of at most NB = 16 or 32
// right-hand-side columns, the batch widths of a sweep step's products and of
// the 2B-wide layer-parallel ones.  Such a product is a stream over the
// operator: every element of A meets all N columns once, 4 N flops per 8
// bytes, so the kernel is built to keep many operator bytes in flight.  A CTA
// of NW_WPC warps owns 32 rows of one problem (lane = row) and one K slice of
// the K blocks of both operand pairs laid end to end; its warps take the
// slice's blocks of NW_KB in turn.  Each warp runs its own ring of NW_NS
// stages filled by asynchronous copies (A block 32 x NW_KB, row-padded, and
// the X block NW_KB x NB), NW_NS - 1 blocks ahead of its products; A is read
// back along the lane's row and X as 16-byte broadcasts.  The warps' partial
// sums are added in warp order; with several K slices per tile (S > 1) the
// last slice to finish adds the slices' sums in slice order (deterministic)
// and re-arms the tile's counter.
template <int NB> __host__ __device__ constexpr int nw_stages() { return 2; }
template <int NB> __host__ __device__ constexpr int nw_stage_elems() { return 32 * (NW_KB + 1) + NW_KB * NB; }
template <int NB> constexpr size_t nw_smem() {
    return sizeof(float2) * (size_t)NW_WPC * nw_stages<NB>() * nw_stage_elems<NB>();
}

// One work unit of the narrow GEMM: tile `tile` (32 rows) of problem *prob, K slice sp
// of S.  PERSIST: called repeatedly by the CTAs of the persistent sweep kernel, whose
// phases read what other CTAs of the same launch wrote, so the right-hand-side blocks
// and the accumulated outputs are read past L1 (16-byte cp.async.cg, ld.global.cg);
// otherwise one unit per CTA, with programmatic dependent launch.
template <int NB, bool PERSIST>
__device__ __forceinline__ void narrow_unit(const GemmProb<float2> *__restrict__ prob, int tile, int sp, int S,
                                            float2 *ws, int *cnt, long long slot, GemmProb<float2> &P, int &last,
                                            unsigned char *nsm) {
    constexpr int NS = nw_stages<NB>(), STG = nw_stage_elems<NB>(), ASZ = 32 * (NW_KB + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float2 *wb = reinterpret_cast<float2 *>(nsm) + warp * NS * STG;
    static_assert(sizeof(GemmProb<float2>) % 8 == 0, "problem descriptor copied as 8-byte words");
    __syncthreads();  // the previous unit of this CTA is done with P and the rings
    for (int w = tid; w < (int)(sizeof(GemmProb<float2>) / 8); w += NW_WPC * 32)
        reinterpret_cast<long long *>(&P)[w] = reinterpret_cast<const long long *>(prob)[w];
    __syncthreads();
    const int M = P.M, N = P.N;
    const int m0 = tile * 32;
    if (m0 >= M) return;  // uniform over the CTA and over the tile's slices
    const int K1 = max(P.K, 0), K2 = max(P.K2, 0);
    const int nb1 = (K1 + NW_KB - 1) / NW_KB, nbt = nb1 + (K2 + NW_KB - 1) / NW_KB;
    const int bps = (nbt + S - 1) / S, b0 = min(nbt, sp * bps), b1 = min(nbt, b0 + bps);
    const int nmine = b1 - b0 > warp ? (b1 - b0 - warp + NW_WPC - 1) / NW_WPC : 0;
    const int ak = lane & 15, ah = lane >> 4;  // A copies: column ak of rows 2 i + ah
    auto issue = [&](int t, int parts) {  // parts: 1 = A block, 2 = X block
        float2 *As = wb + (t % NS) * STG, *Xs = As + ASZ;
        const int b = b0 + warp + t * NW_WPC;
        const bool p2 = b >= nb1;
        const int k0 = (p2 ? b - nb1 : b) * NW_KB, K = p2 ? K2 : K1;
        const float2 *A = p2 ? P.A2 : P.A;
        const long long lda = p2 ? P.lda2 : P.lda;
        const int xseg = p2 ? P.xseg2 : P.xseg;
        const long long ldx = p2 ? P.ldx2 : P.ldx;
        const float2 *const *Xp = p2 ? P.X2 : P.X;
        const int gk = k0 + ak;
        const bool kin = gk < K;
        if (parts & 1) {
#pragma unroll
            for (int i = 0; i < 16; i++) {
                const int r = 2 * i + ah, gm = m0 + r;
                const bool ok = kin && gm < M;
                gemm_cp<8>(As + r * (NW_KB + 1) + ak, ok ? A + (long long)gm * lda + gk : A, ok ? 8u : 0u);
            }
        }
        if (!(parts & 2)) return;
        const bool one = xseg >= K;  // a single segment: no division
        if constexpr (PERSIST) {  // 16-byte copies of column pairs (N and ldx even, 16-byte aligned rows)
#pragma unroll
            for (int q = 0; q < NB / 4; q++) {
                const int e = lane + 32 * q, xr = e / (NB / 2), xc = 2 * (e % (NB / 2)), gx = k0 + xr;
                const bool ok = gx < K && xc < N;
                const float2 *src = A;
                if (ok) {
                    const int sg = one ? 0 : gx / xseg;
                    src = Xp[sg] + (long long)(gx - sg * xseg) * ldx + xc;
                }
                gemm_cp16cg(Xs + xr * NB + xc, src, ok ? 16u : 0u);
            }
            return;
        }
#pragma unroll
        for (int q = 0; q < NB / 2; q++) {
            const int e = lane + 32 * q, xr = e / NB, xc = e % NB, gx = k0 + xr;
            const bool ok = gx < K && xc < N;
            const float2 *src = A;
            if (ok) {
                const int sg = one ? 0 : gx / xseg;
                src = Xp[sg] + (long long)(gx - sg * xseg) * ldx + xc;
            }
            gemm_cp<8>(Xs + xr * NB + xc, src, ok ? 8u : 0u);
        }
    };
    float2 acc[NB];
#pragma unroll
    for (int n = 0; n < NB; n++) acc[n] = czero<float2>();
    // prologue: the operator blocks of the first NS - 1 steps, then (once the kernels this
    // one depends on are complete and visible) their right-hand-side blocks
#pragma unroll
    for (int t = 0; t < NS - 1; t++)
        if (t < nmine) issue(t, 1);
    if constexpr (!PERSIST) asm volatile("griddepcontrol.wait;" ::: "memory");
#pragma unroll
    for (int t = 0; t < NS - 1; t++) {
        if (t < nmine) issue(t, 2);
        gemm_cp_commit();
    }
    for (int t = 0; t < nmine; t++) {
        gemm_cp_wait<NS - 2>();  // this lane's copies of block t have landed
        __syncwarp();            // every lane's have; every lane is done with block t - 1
        if (t + NS - 1 < nmine) issue(t + NS - 1, 3);  // into the stage of block t - 1
        gemm_cp_commit();
        const float2 *As = wb + (t % NS) * STG + lane * (NW_KB + 1), *Xs = wb + (t % NS) * STG + ASZ;
#pragma unroll 4
        for (int kk = 0; kk < NW_KB; kk++) {
            const float2 a = As[kk];
#pragma unroll
            for (int n = 0; n < NB; n += 2) {
                const Pair<float2> x = ld_pair(Xs + kk * NB + n);
                cmac(acc[n], a, x.a);
                cmac(acc[n + 1], a, x.b);
            }
        }
    }
    gemm_cp_wait<0>();
    __syncthreads();  // every warp is done with its ring: it holds the partial sums now
    float2 *red = reinterpret_cast<float2 *>(nsm);  // [warp][32 rows][NB + 1]
#pragma unroll
    for (int n = 0; n < NB; n++) red[(warp * 32 + lane) * (NB + 1) + n] = acc[n];
    __syncthreads();
    if (S > 1) {
        float2 *mine = ws + (slot * S + sp) * (32 * NB);
        for (int e = tid; e < 32 * NB; e += NW_WPC * 32) {
            const int r = e / NB, n = e % NB;
            float2 v = red[r * (NB + 1) + n];
#pragma unroll
            for (int w = 1; w < NW_WPC; w++) v = v + red[(w * 32 + r) * (NB + 1) + n];
            mine[e] = v;
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) last = atomicAdd(&cnt[slot], 1) == S - 1;
        __syncthreads();
        if (!last) return;
        __threadfence();
    }
    const float al = P.alpha;
    for (int e = tid; e < 32 * NB; e += NW_WPC * 32) {
        const int r = e / NB, n = e % NB, m = m0 + r;
        if (m >= M || n >= N) continue;
        float2 v;
        if (S > 1) {
            v = czero<float2>();
            for (int q = 0; q < S; q++) {
                const float2 w = __ldcg(ws + (slot * S + q) * (32 * NB) + e);
                v.x += w.x;
                v.y += w.y;
            }
        } else {
            v = red[r * (NB + 1) + n];
#pragma unroll
            for (int w = 1; w < NW_WPC; w++) v = v + red[(w * 32 + r) * (NB + 1) + n];
        }
        v.x *= al;
        v.y *= al;
        const int sg = m / P.yseg;
        float2 *row = P.Y[sg] + (long long)(m - sg * P.yseg) * P.ldy;
        row[n] = P.beta ? __ldcg(row + n) + v : v;
    }
    if (S > 1 && tid == 0) cnt[slot] = 0;
}

template <int NB>
__global__ void __launch_bounds__(NW_WPC * 32) k_gemm_narrow(const GemmProb<float2> *__restrict__ probs, int S,
                                                             float2 *ws, int *cnt, int max_tiles) {
    __shared__ GemmProb<float2> P;
    __shared__ int last;
    extern __shared__ __align__(16) unsigned char nsm[];
    // programmatic dependent launch: the next kernel may start its own prologue now; this
    // one reads only constant data (descriptors, operators) before griddepcontrol.wait
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int tile = blockIdx.x / S, sp = blockIdx.x % S;
    narrow_unit<NB, false>(probs + blockIdx.y, tile, sp, S, ws, cnt, (long long)blockIdx.y * max_tiles + tile, P,
                           last, nsm);
}

template <int NB>
static void launch_narrow_cfg(const GemmProb<float2> *d_probs, int nprob, int max_tiles, int split, float2 *ws,
                              int *cnt, cudaStream_t st) {
    const size_t sm = nw_smem<NB>();
    static bool attr = false;
    if (!attr) {
        HZ_CU(cudaFuncSetAttribute(k_gemm_narrow<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        attr = true;
    }
    static const bool pdl = !getenv("HZ_PDL") || strcmp(getenv("HZ_PDL"), "0") != 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(max_tiles * split, nprob);
    cfg.blockDim = dim3(NW_WPC * 32);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    HZ_CU(cudaLaunchKernelEx(&cfg, k_gemm_narrow<NB>, d_probs, split, ws, cnt, max_tiles));
}

void launch_gemm_narrow(const GemmProb<float2> *d_probs, int nprob, int max_tiles, int nmax, int split, float2 *ws,
                        int *cnt, cudaStream_t st, int *nl) {
    if (nprob <= 0 || max_tiles <= 0) return;
    if (nmax > NW_NB) throw HzError(HZ_EINVAL, "narrow GEMM: too many columns");
    if (split < 1 || split > 8 || (split > 1 && (!ws || !cnt || (long long)nprob * max_tiles * split > NW_WS_SLOTS)))
        throw HzError(HZ_EINVAL, "narrow GEMM: bad split-K workspace");
    if (nmax <= 8)  // e.g. a batch of 16 solved as two groups of 8 on two streams
        launch_narrow_cfg<8>(d_probs, nprob, max_tiles, split, ws, cnt, st);
    else
        launch_narrow_cfg<NW_NB>(d_probs, nprob, max_tiles, split, ws, cnt, st);
    HZ_CU(cudaGetLastError());
    if (nl) (*nl)++;
}

int gemm_tiles(int M, int N, int cfg) {
    const int bm = cfg == 1 ? 32 : 64, bn = cfg == 2 ? 16 : 32;
    return ((M + bm - 1) / bm) * ((N + bn - 1) / bn);
}

template <class T2, int BM, int BN>
static void launch_gemm_cfg(const GemmProb<T2> *d_probs, int nprob, int max_tiles, int split, T2 *ws, int *cnt,
                            cudaStream_t st) {
    dim3 grid(max_tiles * split, nprob);
    const size_t sm = sizeof(T2) * gemm_stages<T2>() * GBK * (BM + 1 + BN);
    static bool attr = false;
    if (!attr) {
        HZ_CU(cudaFuncSetAttribute(k_gemm<T2, BM, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        attr = true;
    }
    k_gemm<T2, BM, BN><<<grid, 256, sm, st>>>(d_probs, split, ws, cnt, max_tiles);
}

template <class T2>
void launch_gemm(const GemmProb<T2> *d_probs, int nprob, int max_tiles, int split, T2 *ws, int *cnt,
                 cudaStream_t st, int *nl, int cfg) {
    if (nprob <= 0 || max_tiles <= 0) return;
    if (split < 1 || (split > 1 && (!ws || !cnt))) throw HzError(HZ_EINVAL, "batched GEMM: bad split-K workspace");
    if (cfg == 1)
        launch_gemm_cfg<T2, 32, 32>(d_probs, nprob, max_tiles, split, ws, cnt, st);
    else if (cfg == 2)
        launch_gemm_cfg<T2, 64, 16>(d_probs, nprob, max_tiles, split, ws, cnt, st);
    else
        launch_gemm_cfg<T2, 64, 32>(d_probs, nprob, max_tiles, split, ws, cnt, st);
    HZ_CU(cudaGetLastError());
    if (nl) (*nl)++;
}
template void launch_gemm<double2>(const GemmProb<double2> *, int, int, int, double2 *, int *, cudaStream_t, int *,
                                   int);
template void launch_gemm<float2>(const GemmProb<float2> *, int, int, int, float2 *, int *, cudaStream_t, int *, int);

// ========================================================= cell chain ===
// Solve H^{l,c} x = g for every cell and RHS group.  H^{l,c} is block
// tridiagonal over grid rows with diagonal couplings cz between rows; with
// W_j the inverse of the j-th Schur complement:
//   y_0 = W_0 g_0,  y_j = W_j (g_j - cz_{j-1} . y_{j-1})
//   x_{nz-1} = y_{nz-1},  x_j = y_j - W_j (cz_j . x_{j+1})
// One CTA per (cell, NT columns).  The W blocks are streamed through a
// ST-stage ring of CH-row chunks with cp.async; the chunk sequence (forward
// W_0..W_{nz-1}, then backward W_{nz-2}..W_0) is known in advance, so the
// prefetch runs ahead across step boundaries.  Each thread owns a
// (CH/16) x (NT/16) tile of complex outputs.
// vol layout: [cell vol_off + jz*nx + jx][B] (RHS innermost), in place.
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

template <class T2, int NT, int CH, int ST>
__global__ void __launch_bounds__(256) k_cell_chain(const CellDesc *__restrict__ cells, const T2 *__restrict__ W,
                                                    const T2 *__restrict__ cz, T2 *vol, int B) {
    constexpr int TM = CH / 16, TN = NT / 16;
    constexpr int GP = 16;  // register-prefetch slots per thread for the next step's global vector
    extern __shared__ __align__(16) unsigned char smraw[];
    const CellDesc cd = cells[blockIdx.y];  // fields in registers
    const int nx = cd.nx, nz = cd.nz, ldw = cd.ldw;
    const int n0 = blockIdx.x * NT;
    if (n0 >= B) return;
    T2 *tbuf0 = reinterpret_cast<T2 *>(smraw);  // t of the current step
    T2 *tbuf1 = tbuf0 + nx * NT;                // t of the next step (built by the epilogue)
    T2 *gb = tbuf1 + nx * NT;                   // global vector used by this step's epilogue
    T2 *ring = gb + nx * NT;
    const int tid = threadIdx.x, rg = tid >> 4, cg = tid & 15;
    const int nch = (nx + CH - 1) / CH;
    const int nsteps = 2 * nz - 1;
    const int total = nsteps * nch;
    const T2 *Wc = W + cd.w_off;
    const T2 *czc = cz + cd.cz_off;
    T2 *v = vol + cd.vol_off * (long long)B;
    const long long rs = (long long)nx * B;
    auto jb_of = [&](int s) { return s < nz ? s : 2 * nz - 2 - s; };
    auto issue = [&](int q) {
        if (q < total) {
            const int s = q / nch, c = q % nch;
            const int jb = jb_of(s);
            const int rows = min(CH, nx - c * CH);
            const char *src = reinterpret_cast<const char *>(Wc + (long long)jb * nx * ldw + (long long)c * CH * ldw);
            char *dst = reinterpret_cast<char *>(ring + (q % ST) * CH * ldw);
            const int nbytes = rows * ldw * (int)sizeof(T2);
            for (int off = tid * 16; off < nbytes; off += 256 * 16) cp_async16(dst + off, src + off);
        }
        cp_async_commit();
    };
    // the global vector an epilogue needs: forward step s -> g of step s+1 (to form t_{s+1});
    // backward step s -> y of step s (x = y - W t).  Both live at v + jb*rs.
    auto gvec_step = [&](int s) -> int {
        if (s < nz - 1) return s + 1;  // forward, next forward step's source
        if (s < nz) return -1;         // last forward step: t of the first backward step needs no global data
        return s;                      // backward: its own y
    };
    const int nel = nx * NT;
    const bool gp_ok = nel <= 256 * GP;
    T2 greg[GP];
    auto gprefetch = [&](int s) {
        const int sg = (s < nsteps) ? gvec_step(s) : -1;
        if (sg < 0) return;
        const T2 *src = v + jb_of(sg) * rs;
        if (gp_ok) {
#pragma unroll
            for (int i = 0; i < GP; i++) {
                const int e = tid + 256 * i;
                if (e < nel) {
                    const int jx = e / NT, nn = e % NT;
                    greg[i] = (n0 + nn < B) ? src[(long long)jx * B + n0 + nn] : czero<T2>();
                }
            }
        }
    };
    auto gstage = [&](int s) {  // registers (or global) -> gb
        const int sg = (s < nsteps) ? gvec_step(s) : -1;
        if (sg < 0) return;
        if (gp_ok) {
#pragma unroll
            for (int i = 0; i < GP; i++) {
                const int e = tid + 256 * i;
                if (e < nel) gb[e] = greg[i];
            }
        } else {
            const T2 *src = v + jb_of(sg) * rs;
            for (int e = tid; e < nel; e += 256) {
                const int jx = e / NT, nn = e % NT;
                gb[e] = (n0 + nn < B) ? src[(long long)jx * B + n0 + nn] : czero<T2>();
            }
        }
    };
#pragma unroll
    for (int q = 0; q < ST - 1; q++) issue(q);
    // t_0 = g_0
    for (int e = tid; e < nel; e += 256) {
        const int jx = e / NT, nn = e % NT;
        tbuf0[e] = (n0 + nn < B) ? v[(long long)jx * B + n0 + nn] : czero<T2>();
    }
    gprefetch(0);
    int q = 0;
    T2 *tc = tbuf0, *tn = tbuf1;
    for (int s = 0; s < nsteps; s++) {
        const bool fwd = s < nz;
        const int jb = jb_of(s);
        if (s > 0) __syncthreads();  // previous step's epilogues done (gb, t of this step complete)
        gstage(s);                   // gb for this step's epilogue
        __syncthreads();
        gprefetch(s + 1);  // in flight during this step
        T2 *g = v + jb * rs;
        for (int c = 0; c < nch; c++, q++) {
            cp_async_wait<ST - 2>();
            __syncthreads();  // chunk q visible; chunk q-1's slot no longer read
            issue(q + ST - 1);
            const T2 *Wq = ring + (q % ST) * CH * ldw;
            T2 acc[TM][TN];
#pragma unroll
            for (int i = 0; i < TM; i++)
#pragma unroll
                for (int t = 0; t < TN; t++) acc[i][t] = czero<T2>();
            const T2 *wr = Wq + (rg * TM) * ldw;
            if constexpr (TN % 2 == 0) {
                // columns 2cg, 2cg+1 (+32 per extra pair): 16-byte loads of adjacent
                // columns and of W(k), W(k+1)
                const T2 *xr = tc + 2 * cg;
                const T2 *wp[TM];
#pragma unroll
                for (int i = 0; i < TM; i++) wp[i] = wr + i * ldw;
                int k = 0;
#pragma unroll 2
                for (; k + 1 < nx; k += 2) {
                    Pair<T2> w[TM];
#pragma unroll
                    for (int i = 0; i < TM; i++) w[i] = ld_pair(wp[i] + k);
                    const T2 *xk = xr + k * NT;
#pragma unroll
                    for (int tp = 0; tp < TN / 2; tp++) {
                        const Pair<T2> x0 = ld_pair(xk + 32 * tp);
                        const Pair<T2> x1 = ld_pair(xk + NT + 32 * tp);
#pragma unroll
                        for (int i = 0; i < TM; i++) {
                            cmac(acc[i][2 * tp], w[i].a, x0.a);
                            cmac(acc[i][2 * tp + 1], w[i].a, x0.b);
                            cmac(acc[i][2 * tp], w[i].b, x1.a);
                            cmac(acc[i][2 * tp + 1], w[i].b, x1.b);
                        }
                    }
                }
                if (k < nx) {
#pragma unroll
                    for (int tp = 0; tp < TN / 2; tp++) {
                        const Pair<T2> x0 = ld_pair(xr + k * NT + 32 * tp);
#pragma unroll
                        for (int i = 0; i < TM; i++) {
                            cmac(acc[i][2 * tp], wr[i * ldw + k], x0.a);
                            cmac(acc[i][2 * tp + 1], wr[i * ldw + k], x0.b);
                        }
                    }
                }
            } else {
                const T2 *xr = tc + cg;
                for (int k = 0; k < nx; k++) {
                    T2 a[TM], xv[TN];
#pragma unroll
                    for (int i = 0; i < TM; i++) a[i] = wr[i * ldw + k];
#pragma unroll
                    for (int t = 0; t < TN; t++) xv[t] = xr[k * NT + 16 * t];
#pragma unroll
                    for (int i = 0; i < TM; i++)
#pragma unroll
                        for (int t = 0; t < TN; t++) cmac(acc[i][t], a[i], xv[t]);
                }
            }
            // epilogue: this step's output and the next step's t
#pragma unroll
            for (int i = 0; i < TM; i++) {
                const int m = c * CH + rg * TM + i;
                if (m >= nx) continue;
#pragma unroll
                for (int t = 0; t < TN; t++) {
                    const int nn = (TN % 2 == 0) ? 2 * cg + (t & 1) + 32 * (t >> 1) : cg + 16 * t;
                    const bool live = n0 + nn < B;
                    T2 out = acc[i][t], tnext;
                    if (fwd) {
                        if (s + 1 < nz)
                            tnext = gb[m * NT + nn] - czc[(long long)jb * nx + m] * out;  // g_{j+1} - c_j y_j
                        else if (jb > 0)
                            tnext = czc[(long long)(jb - 1) * nx + m] * out;  // first backward: c_{nz-2} x_{nz-1}
                        else
                            tnext = czero<T2>();
                    } else {
                        out = gb[m * NT + nn] - out;  // x_j = y_j - W_j t
                        tnext = (jb > 0) ? czc[(long long)(jb - 1) * nx + m] * out : czero<T2>();
                    }
                    if (!live) {
                        out = czero<T2>();
                        tnext = czero<T2>();
                    }
                    tn[m * NT + nn] = tnext;
                    if (live) g[(long long)m * B + n0 + nn] = out;
                }
            }
        }
        T2 *tt = tc;
        tc = tn;
        tn = tt;
    }
    cp_async_wait<0>();
}

// FP32 cell chain for panels of at most 16 right-hand sides (the batch of the
// 2000 x 4000 workload): the same recurrence as k_cell_chain, laid out for the
// FMA pipes.  A thread owns TM rows x 2 adjacent columns of each 64-row chunk, so
// a pair of K steps costs TM 16-byte loads of W (its rows, k and k+1) and two of
// t (columns 2c, 2c+1 at k and k+1) per 16 TM FMAs; the W rows in the two-stage ring
// are padded by one 16-byte unit so that the four row groups of a warp fall in
// distinct banks.  The epilogue's operands (next source / own y, and the z
// coupling) are loaded into registers one step ahead, in the thread's own output
// layout, right after the epilogue that consumed the previous ones.
constexpr int C16_CH = 64, C16_MAXCH = 3;  // chunk rows; chunks per step (nx <= 192)
__host__ __device__ constexpr size_t c16_smem(int ldws, int max_nx) {
    return sizeof(float2) * ((size_t)2 * C16_CH * ldws + (size_t)2 * max_nx * 16);
}
template <int TM>
__global__ void __launch_bounds__(512 / TM, 1) k_cell_chain16(const CellDesc *__restrict__ cells,
                                                              const float2 *__restrict__ W,
                                                              const float2 *__restrict__ cz, float2 *vol, int B,
                                                              int ldws) {
    constexpr int NTH = 512 / TM;  // threads: 8 column pairs x (64 / TM) row groups
    extern __shared__ __align__(16) unsigned char smraw[];
    const CellDesc cd = cells[blockIdx.y];
    const int nx = cd.nx, nz = cd.nz, ldw = cd.ldw;
    const int n0 = blockIdx.x * 16;
    if (n0 >= B) return;
    float2 *ring = reinterpret_cast<float2 *>(smraw);  // 2 stages x 64 rows x ldws
    float2 *tc = ring + 2 * C16_CH * ldws;             // t of the current step [nx][16]
    float2 *tn = tc + nx * 16;                          // t of the next step
    const int tid = threadIdx.x, cg = tid & 7, rg = tid >> 3;
    const int nch = (nx + C16_CH - 1) / C16_CH, nsteps = 2 * nz - 1, total = nsteps * nch;
    const float2 *Wc = W + cd.w_off;
    const float2 *czc = cz + cd.cz_off;
    float2 *v = vol + cd.vol_off * (long long)B;
    const long long rs = (long long)nx * B;
    const int units = ldw / 2;  // 16-byte units per W row
    const float inv_units = 1.0f / (float)units;
    auto jb_of = [&](int s) { return s < nz ? s : 2 * nz - 2 - s; };
    auto issue = [&](int q) {
        if (q < total) {
            const int s = q / nch, c = q % nch;
            const int rows = min(C16_CH, nx - c * C16_CH);
            const float2 *src = Wc + ((long long)jb_of(s) * nx + (long long)c * C16_CH) * ldw;
            float2 *dst = ring + (q & 1) * C16_CH * ldws;
            for (int u = tid; u < rows * units; u += NTH) {
                const int r = __float2int_rz(((float)u + 0.5f) * inv_units), k2 = u - r * units;
                cp_async16(dst + r * ldws + 2 * k2, src + (long long)r * ldw + 2 * k2);
            }
        }
        cp_async_commit();
    };
    // epilogue operands of step s: the global vector (forward: g of step s+1; backward: own y)
    // and the coupling row (forward: c_s, or c_{nz-2} on the last forward step; backward:
    // c_{jb-1}); -1: none
    auto grow = [&](int s) { return s < nz - 1 ? s + 1 : (s < nz ? -1 : jb_of(s)); };
    auto crow = [&](int s) { return s < nz - 1 ? s : (s < nz ? nz - 2 : jb_of(s) - 1); };
    float2 gr[C16_MAXCH][TM][2], cr[C16_MAXCH][TM];
    auto prefetch = [&](int s, int c) {  // operands of chunk c of step s
        if (s >= nsteps) return;
        const int gs = grow(s), cs = crow(s);
#pragma unroll
        for (int i = 0; i < TM; i++) {
            const int m = c * C16_CH + rg * TM + i;
            const bool mok = m < nx;
            cr[c][i] = (mok && cs >= 0) ? czc[(long long)cs * nx + m] : czero<float2>();
#pragma unroll
            for (int t = 0; t < 2; t++) {
                const int nn = 2 * cg + t;
                gr[c][i][t] = (mok && gs >= 0 && n0 + nn < B) ? v[gs * rs + (long long)m * B + n0 + nn] : czero<float2>();
            }
        }
    };
    issue(0);
    for (int e = tid; e < nx * 16; e += NTH) {  // t_0 = g_0
        const int jx = e >> 4, nn = e & 15;
        tc[e] = (n0 + nn < B) ? v[(long long)jx * B + n0 + nn] : czero<float2>();
    }
#pragma unroll
    for (int c = 0; c < C16_MAXCH; c++)
        if (c < nch) prefetch(0, c);
    int q = 0;
    for (int s = 0; s < nsteps; s++) {
        const bool fwd = s < nz;
        const int jb = jb_of(s);
        float2 *g = v + jb * rs;
#pragma unroll
        for (int c = 0; c < C16_MAXCH; c++) {
            if (c >= nch) break;
            cp_async_wait<0>();
            __syncthreads();  // chunk q landed for all; chunk q-1 and the previous step's t are done
            issue(q + 1);     // into the other stage
            const float2 *w0 = ring + (q & 1) * C16_CH * ldws + (rg * TM) * ldws;
            const float2 *xr = tc + 2 * cg;
            float2 acc[TM][2];
#pragma unroll
            for (int i = 0; i < TM; i++) acc[i][0] = acc[i][1] = czero<float2>();
            // K pairs software-pipelined: the next pair's shared-memory loads are issued before
            // the current pair's FMAs; even and odd K accumulate apart (shorter FMA chains)
            float2 acc2[TM][2];
#pragma unroll
            for (int i = 0; i < TM; i++) acc2[i][0] = acc2[i][1] = czero<float2>();
            int k = 0;
            const int kp = nx & ~1;  // K covered by pairs
            if (kp > 0) {
                Pair<float2> x0 = ld_pair(xr), x1 = ld_pair(xr + 16), p[TM];
#pragma unroll
                for (int i = 0; i < TM; i++) p[i] = ld_pair(w0 + i * ldws);
#pragma unroll 2
                for (; k + 2 < kp; k += 2) {
                    const Pair<float2> y0 = ld_pair(xr + (k + 2) * 16), y1 = ld_pair(xr + (k + 3) * 16);
                    Pair<float2> pn[TM];
#pragma unroll
                    for (int i = 0; i < TM; i++) pn[i] = ld_pair(w0 + i * ldws + k + 2);
#pragma unroll
                    for (int i = 0; i < TM; i++) {
                        cmac(acc[i][0], p[i].a, x0.a);
                        cmac(acc[i][1], p[i].a, x0.b);
                        cmac(acc2[i][0], p[i].b, x1.a);
                        cmac(acc2[i][1], p[i].b, x1.b);
                        p[i] = pn[i];
                    }
                    x0 = y0;
                    x1 = y1;
                }
#pragma unroll
                for (int i = 0; i < TM; i++) {  // the last pair
                    cmac(acc[i][0], p[i].a, x0.a);
                    cmac(acc[i][1], p[i].a, x0.b);
                    cmac(acc2[i][0], p[i].b, x1.a);
                    cmac(acc2[i][1], p[i].b, x1.b);
                }
                k = kp;
            }
#pragma unroll
            for (int i = 0; i < TM; i++) {
                acc[i][0] = acc[i][0] + acc2[i][0];
                acc[i][1] = acc[i][1] + acc2[i][1];
            }
            if (k < nx) {
                const Pair<float2> x0 = ld_pair(xr + k * 16);
#pragma unroll
                for (int i = 0; i < TM; i++) {
                    const float2 w = w0[i * ldws + k];
                    cmac(acc[i][0], w, x0.a);
                    cmac(acc[i][1], w, x0.b);
                }
            }
#pragma unroll
            for (int i = 0; i < TM; i++) {
                const int m = c * C16_CH + rg * TM + i;
                if (m >= nx) continue;
#pragma unroll
                for (int t = 0; t < 2; t++) {
                    const int nn = 2 * cg + t;
                    const bool live = n0 + nn < B;
                    float2 out = acc[i][t], tnext;
                    if (fwd) {
                        if (s + 1 < nz)
                            tnext = gr[c][i][t] - cr[c][i] * out;  // g_{j+1} - c_j y_j
                        else
                            tnext = (jb > 0) ? cr[c][i] * out : czero<float2>();  // first backward: c_{nz-2} x_{nz-1}
                    } else {
                        out = gr[c][i][t] - out;  // x_j = y_j - W_j t
                        tnext = (jb > 0) ? cr[c][i] * out : czero<float2>();
                    }
                    if (!live) {
                        out = czero<float2>();
                        tnext = czero<float2>();
                    }
                    tn[m * 16 + nn] = tnext;
                    if (live) g[(long long)m * B + n0 + nn] = out;
                }
            }
            prefetch(s + 1, c);  // in flight until this chunk's epilogue of the next step
            q++;
        }
        float2 *tt = tc;
        tc = tn;
        tn = tt;
    }
    cp_async_wait<0>();
}

static bool cell_chain16(const CellDesc *d_cells, int ncell, const float2 *W, const float2 *cz, float2 *vol, int B,
                         int max_nx, cudaStream_t st) {
    if (B > 16 || max_nx > C16_CH * C16_MAXCH) return false;
    const int ldws = ((max_nx + 1) & ~1) + 2;
    const size_t sm = c16_smem(ldws, max_nx);
    if (sm > 227 * 1024) return false;
    // two rows per thread (256 threads); one row per thread with 512 threads measured 33 %
    // slower on the 2000 x 4000 workload (more shared-memory loads per FMA)
    static size_t attr = 0;
    if (sm > attr) {
        HZ_CU(cudaFuncSetAttribute(k_cell_chain16<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        attr = sm;
    }
    k_cell_chain16<2><<<dim3(1, ncell), 256, sm, st>>>(d_cells, W, cz, vol, B, ldws);
    HZ_CU(cudaGetLastError());
    return true;
}

template <class T2, int NT, int CH, int ST>
static bool cell_chain_cfg(const CellDesc *d_cells, int ncell, const T2 *W, const T2 *cz, T2 *vol, int B, int max_nx,
                           cudaStream_t st) {
    const int ldw = (max_nx + 1) & ~1;
    const size_t sm = (size_t)(3 * max_nx * NT + ST * CH * ldw) * sizeof(T2);
    if (sm > 220 * 1024) return false;
    HZ_CU(cudaFuncSetAttribute(k_cell_chain<T2, NT, CH, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    dim3 grid((B + NT - 1) / NT, ncell);
    k_cell_chain<T2, NT, CH, ST><<<grid, 256, sm, st>>>(d_cells, W, cz, vol, B);
    HZ_CU(cudaGetLastError());
    return true;
}

template <class T2>
void launch_cell_chain(const CellDesc *d_cells, int ncell, const T2 *W, const T2 *cz, T2 *vol, int B, int max_nx,
                       cudaStream_t st, int *nl) {
    if (ncell <= 0 || B <= 0) return;
    // widest RHS tile that fits; narrow tiles when few cells would leave SMs idle
    bool ok = false;
    if constexpr (std::is_same<T2, float2>::value) {
        static const bool c16 = !getenv("HZ_CELL") || strcmp(getenv("HZ_CELL"), "tiled") != 0;
        if (c16 && B <= 16 && cell_chain16(d_cells, ncell, W, cz, vol, B, max_nx, st)) {
            if (nl) (*nl)++;
            return;
        }
    }
    if (B > 16) ok = cell_chain_cfg<T2, 32, 64, 2>(d_cells, ncell, W, cz, vol, B, max_nx, st);
    if (!ok && B > 16) ok = cell_chain_cfg<T2, 32, 32, 3>(d_cells, ncell, W, cz, vol, B, max_nx, st);
    if (!ok) ok = cell_chain_cfg<T2, 16, 32, 3>(d_cells, ncell, W, cz, vol, B, max_nx, st);
    if (!ok) ok = cell_chain_cfg<T2, 16, 16, 2>(d_cells, ncell, W, cz, vol, B, max_nx, st);
    if (!ok) throw HzError(HZ_ENOMEM, "cell solve: cell too wide for shared memory");
    if (nl) (*nl)++;
}
template void launch_cell_chain<double2>(const CellDesc *, int, const double2 *, const double2 *, double2 *, int,
                                         int, cudaStream_t, int *);
template void launch_cell_chain<float2>(const CellDesc *, int, const float2 *, const float2 *, float2 *, int, int,
                                        cudaStream_t, int *);

// ======================================================== inner sweep ===
// Block-LU sweeps of a layer's inner SIE (Section 4.2.2) with inverted diagonal
// blocks.  With h_j = W_j g_j computed beforehand for every interface (one
// batched product) and P_j = W_j(:, 0:nz) Z_j precomputed offline, both sweeps
// are the recurrence
//   forward : y_0 = h_0,        y_j = h_j + P_j y_{j-1}   (j = 1..J-1)
//   backward: x_{J-1} = y_{J-1}, x_j = y_j + V_j x_{j+1}   (j = J-2..0)
// One thread-block cluster of R CTAs runs the recurrence of one layer for a
// tile of right-hand sides.  CTA r owns a slab of rows of every Q_j and of z_j;
// each step it computes its rows of z_j from the whole z_{j-1} held in its
// shared memory, stores them to global memory and pushes them into the shared
// memory of every CTA of the cluster (distributed shared memory), where they
// complete a transaction-count mbarrier.  Every wait is bounded: a CTA that
// gives up sets the error word (HZ_ETIMEOUT on the host) and the kernel still
// ends.
// Layout: slot j+1 of the layer's inner buffer holds interface j ([2nz][B]).
// shared-memory / cluster helpers (inline PTX)
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned cluster_map(unsigned addr, int rank) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
__device__ __forceinline__ void mbar_init(unsigned mb, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(unsigned mb, unsigned tx) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(tx) : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned mb, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mb), "r"(parity)
        : "memory");
    return ok != 0;
}
// bulk copy of `bytes` from this CTA's shared memory to another CTA of the
// cluster, completing on that CTA's mbarrier
__device__ __forceinline__ void bulk_to_peer(unsigned dst_cluster, unsigned src_cta, unsigned bytes,
                                             unsigned mbar_cluster) {
    asm volatile(
        "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst_cluster),
        "r"(src_cta), "r"(bytes), "r"(mbar_cluster)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_acq_cluster(unsigned mb, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mb), "r"(parity)
        : "memory");
    return ok != 0;
}
// bulk (TMA) copy global -> this CTA's shared memory, completing on its mbarrier
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void *src, unsigned bytes, unsigned mb) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mb)
                 : "memory");
}
// 16-byte store into a CTA of the cluster, completing on that CTA's mbarrier
__device__ __forceinline__ void st_async16(unsigned dst, uint4 v, unsigned mb) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(
                     dst),
                 "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w), "r"(mb)
                 : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
// wait for phase `parity` of an mbarrier for at most the context's wait limit
// (1 ms once the thread has already given up somewhere); on expiry set the
// error word and `dead` and return false
__device__ __forceinline__ bool mbar_wait_bounded(unsigned mb, unsigned parity, bool cluster_scope, bool &dead,
                                                  int *err) {
    const unsigned long long limit_ns = dead ? DRAIN_WAIT_NS : wait_limit_ns(err);
    unsigned long long t0 = 0;
    for (unsigned it = 0;; it++) {
        if (cluster_scope ? mbar_try_acq_cluster(mb, parity) : mbar_try(mb, parity)) return true;
        if ((it & 63u) == 63u) {
            const unsigned long long t = global_ns();
            if (t0 == 0) {
                t0 = t;
            } else if (t - t0 > limit_ns) {
                if (!dead) atomicExch(err, 1);
                dead = true;
                return false;
            }
        }
    }
}

// padded row stride of the Q slab in shared memory (breaks bank aliasing of
// rows that are 2*nz complex apart, keeps 16-byte alignment)
template <class T2> __host__ __device__ inline int q_ld(int n2) { return sizeof(T2) == 8 ? n2 + 2 : n2 + 1; }

// Fallback form for operators whose row slabs do not fit the staged kernel
// below (e.g. FP64 with 2nz' > 256): the Q slab is prefetched through
// registers one step ahead and slabs move between CTAs by bulk copies.
template <class T2, int NB>
__global__ void __launch_bounds__(256) k_inner_sweep_regq(const LayerDesc *__restrict__ layers,
                                                     const int *__restrict__ ids, const T2 *__restrict__ P,
                                                     const T2 *__restrict__ V, const T2 *__restrict__ H, T2 *X,
                                                     int B, int *err) {
    namespace cg = cooperative_groups;
    constexpr int NP = NB / 2;  // column pairs
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ __align__(8) unsigned long long mbar[2];
    cg::cluster_group cl = cg::this_cluster();
    const int R = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const int grp = blockIdx.x / R;
    const LayerDesc ld = layers[ids[blockIdx.y]];  // fields in registers
    const int nz = ld.nz, n2 = 2 * nz, J = ld.C - 1;
    if (J <= 0) return;  // uniform over the cluster
    const int n0 = grp * NB;
    const int rs = (n2 + R - 1) / R;
    const int r0 = min(n2, rank * rs), r1 = min(n2, r0 + rs), nr = r1 - r0;
    const int ldq = q_ld<T2>(n2);
    T2 *zb0 = reinterpret_cast<T2 *>(smraw);
    T2 *zb1 = zb0 + n2 * NB;
    T2 *Qs = zb1 + n2 * NB;
    const long long slot = (long long)n2 * B;
    const T2 *h = H + ld.inner_off * (long long)B;
    T2 *x = X + ld.inner_off * (long long)B;
    const T2 *Pl = P + ld.P_off, *Vl = V + ld.V_off;
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(smem_u32(&mbar[0]), 1);
        mbar_init(smem_u32(&mbar[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int e = tid; e < n2 * NB; e += 256) {
        int k = e / NB, n = e % NB;
        zb0[e] = (n0 + n < B) ? h[slot + (long long)k * B + n0 + n] : czero<T2>();
    }
    for (int e = tid; e < nr * NB; e += 256) {
        int m = r0 + e / NB, n = e % NB;
        if (n0 + n < B) x[slot + (long long)m * B + n0 + n] = h[slot + (long long)m * B + n0 + n];
    }
    const int S = 2 * (J - 1);
    // thread -> (row m, column pair np, K part kp); K parts are contiguous even-length ranges
    const int outs = nr * NP;
    int ks = 1;
    while (ks < 32 && outs * ks * 2 <= 256) ks *= 2;
    const int per = 256 / ks;
    const bool single = outs <= per;
    // Q slab prefetch: nr rows of n2 complex, as 16-byte vectors (rows are contiguous in global memory)
    constexpr int PF = 12;
    const int vrow = (int)(n2 * sizeof(T2) / 16);  // vectors per row
    const int nvec = nr * vrow;
    const bool use_pf = nvec <= 256 * PF;
    int4 pf[PF];
    auto step_j = [&](int s) { return s < J - 1 ? s + 1 : J - 2 - (s - (J - 1)); };
    auto qptr = [&](int s) -> const T2 * {
        return (s < J - 1 ? Pl : Vl) + (long long)step_j(s) * n2 * n2 + (long long)r0 * n2;
    };
    auto bptr = [&](int s) -> const T2 * { return (s < J - 1 ? h : x) + (long long)(step_j(s) + 1) * slot; };
    const int o_me = tid / ks, kp = tid % ks;
    const int m_me = o_me / NP, np_me = o_me % NP;
    const bool out_me = single && o_me < outs && kp == 0;
    auto prefetch = [&](int s, Pair<T2> &bnext) {
        if (s >= S) return;
        if (use_pf) {
            const int4 *src = reinterpret_cast<const int4 *>(qptr(s));
#pragma unroll
            for (int i = 0; i < PF; i++) {
                int v = tid + 256 * i;
                if (v < nvec) pf[i] = src[v];
            }
        }
        if (out_me) {
            const T2 *bp = bptr(s) + (long long)(r0 + m_me) * B + n0 + 2 * np_me;
            bnext.a = (n0 + 2 * np_me < B) ? bp[0] : czero<T2>();
            bnext.b = (n0 + 2 * np_me + 1 < B) ? bp[1] : czero<T2>();
        }
    };
    auto qstore = [&](const int4 *src) {  // vectors -> padded rows of Qs
        for (int v = tid; v < nvec; v += 256) {
            const int row = v / vrow, col = v % vrow;
            reinterpret_cast<int4 *>(Qs + row * ldq)[col] = src[v];
        }
    };
    Pair<T2> bcur{czero<T2>(), czero<T2>()}, bnext{czero<T2>(), czero<T2>()};
    prefetch(0, bcur);
    cl.sync();  // all CTAs started, mbarriers initialised: peers may copy into us from now on
    const unsigned rx_bytes = (unsigned)((n2 - nr) * NB * sizeof(T2));
    const unsigned my_bytes = (unsigned)(nr * NB * sizeof(T2));
    unsigned ph0 = 0u, ph1 = 0u;
    bool dead = false;
    // CTAs without rows (2nz' < R * rows-per-CTA) neither send nor receive
    for (int s = 0; s < S && nr > 0; s++) {
        const int bo = (s & 1) ^ 1;  // input z_s in zb[s&1], output z_{s+1} into zb[bo]
        T2 *cur = bo ? zb0 : zb1, *nxt = bo ? zb1 : zb0;
        if (use_pf) {
#pragma unroll
            for (int i = 0; i < PF; i++) {
                const int v = tid + 256 * i;
                if (v < nvec) {
                    const int row = v / vrow, col = v % vrow;
                    reinterpret_cast<int4 *>(Qs + row * ldq)[col] = pf[i];
                }
            }
        } else {
            qstore(reinterpret_cast<const int4 *>(qptr(s)));
        }
        if (s > 0) {  // previous step's rows to global memory
            T2 *outp = x + (long long)(step_j(s - 1) + 1) * slot;
            for (int e = tid; e < nr * NB; e += 256) {
                const int m = r0 + e / NB, n = e % NB;
                if (n0 + n < B) outp[(long long)m * B + n0 + n] = cur[m * NB + n];
            }
        }
        __syncthreads();
        prefetch(s + 1, bnext);
        const T2 *base = bptr(s);
        for (int o0 = 0; o0 < outs; o0 += per) {
            const int o = o0 + o_me;
            T2 a0 = czero<T2>(), a1 = czero<T2>(), c0 = czero<T2>(), c1 = czero<T2>();
            const int m = o / NP, np = o % NP;
            if (o < outs) {
                // K interleaved over the ks lanes of an output (adjacent rows of z fall in
                // different banks); z read as 16-byte column pairs
                const T2 *q = Qs + m * ldq;
                const T2 *zc = cur + 2 * np;
                int k = kp;
                for (; k + ks < n2; k += 2 * ks) {
                    const T2 q0 = q[k], q1 = q[k + ks];
                    const Pair<T2> z0 = ld_pair(zc + k * NB);
                    const Pair<T2> z1 = ld_pair(zc + (k + ks) * NB);
                    cmac(a0, q0, z0.a);
                    cmac(a1, q0, z0.b);
                    cmac(c0, q1, z1.a);
                    cmac(c1, q1, z1.b);
                }
                if (k < n2) {
                    const Pair<T2> z0 = ld_pair(zc + k * NB);
                    cmac(a0, q[k], z0.a);
                    cmac(a1, q[k], z0.b);
                }
            }
            T2 acc0 = a0 + c0, acc1 = a1 + c1;
            for (int off = ks >> 1; off > 0; off >>= 1) {
                acc0.x += __shfl_down_sync(0xffffffffu, acc0.x, off);
                acc0.y += __shfl_down_sync(0xffffffffu, acc0.y, off);
                acc1.x += __shfl_down_sync(0xffffffffu, acc1.x, off);
                acc1.y += __shfl_down_sync(0xffffffffu, acc1.y, off);
            }
            if (o < outs && kp == 0) {
                const int n = 2 * np;
                Pair<T2> bv;
                if (single) {
                    bv = bcur;
                } else {
                    const T2 *bp = base + (long long)(r0 + m) * B + n0 + n;
                    bv.a = (n0 + n < B) ? bp[0] : czero<T2>();
                    bv.b = (n0 + n + 1 < B) ? bp[1] : czero<T2>();
                }
                T2 *dst = nxt + (r0 + m) * NB + n;
                dst[0] = (n0 + n < B) ? bv.a + acc0 : czero<T2>();
                dst[1] = (n0 + n + 1 < B) ? bv.b + acc1 : czero<T2>();
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> async-proxy reads
        __syncthreads();  // my slab of z_{s+1} complete
        if (tid == 0) {
            const unsigned mb_local = smem_u32(&mbar[bo]);
            mbar_arrive_tx(mb_local, rx_bytes);
            if (my_bytes > 0) {
                const unsigned src = smem_u32(nxt + r0 * NB);
                for (int d = 0; d < R; d++) {
                    if (d == rank || d * rs >= n2) continue;
                    bulk_to_peer(cluster_map(src, d), src, my_bytes, cluster_map(mb_local, d));
                }
            }
        }
        // wait for every peer's slab (bounded: a timeout sets the error word and the
        // whole CTA leaves the steps together)
        mbar_wait_bounded(smem_u32(&mbar[bo]), bo ? ph1 : ph0, false, dead, err);
        if (bo) ph1 ^= 1u; else ph0 ^= 1u;
        if (__syncthreads_or(dead)) break;
        bcur = bnext;
    }
    if (S > 0 && !dead) {
        const T2 *cur = (S & 1) ? zb1 : zb0;
        T2 *outp = x + (long long)(step_j(S - 1) + 1) * slot;
        for (int e = tid; e < nr * NB; e += 256) {
            const int m = r0 + e / NB, n = e % NB;
            if (n0 + n < B) outp[(long long)m * B + n0 + n] = cur[m * NB + n];
        }
    }
    cl.sync();  // no CTA leaves while peers may still copy into or out of it
    if (__syncthreads_or(dead)) __nanosleep(20000);  // copies a timed-out peer issued may still be landing
}

template <class T2, int NB>
static bool inner_sweep_regq(const LayerDesc *d_layers, const int *ids, int nlayer, const T2 *P, const T2 *V,
                           const T2 *H, T2 *X, int B, int max_n2, int *err, cudaStream_t st) {
    const int groups = (B + NB - 1) / NB;
    auto smem = [&](int R) {
        return (size_t)(2 * max_n2 * NB + ((max_n2 + R - 1) / R) * q_ld<T2>(max_n2)) * sizeof(T2);
    };
    // smallest cluster whose row slab fits in shared memory
    int Rmin = 1;
    while (Rmin <= 16 && smem(Rmin) > 220 * 1024) Rmin *= 2;
    if (Rmin > 16) return false;
    // preferred: the largest cluster (smallest row slab per CTA, so the
    // slab fits the register prefetch and each step's dot products are short)
    int R = 16;
    auto kern = k_inner_sweep_regq<T2, NB>;
    HZ_CU(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    cfg.blockDim = dim3(256, 1, 1);
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // largest cluster the device can co-schedule
    for (; R >= Rmin; R /= 2) {
        cfg.dynamicSmemBytes = smem(R);
        HZ_CU(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.dynamicSmemBytes));
        attr[0].val.clusterDim.x = R;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(R * groups, nlayer, 1);
        int ncl = 0;
        if (cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg) == cudaSuccess && ncl > 0) break;
        cudaGetLastError();
    }
    if (R < Rmin) return false;
    HZ_CU(cudaLaunchKernelEx(&cfg, kern, d_layers, ids, P, V, H, X, B, err));
    return true;
}


// 16-byte chunks of complex values: two float2 or one double2
template <class T2> struct Chunk16;
template <> struct Chunk16<float2> {
    static constexpr int n = 2;
    __device__ static void load(const float2 *p, float2 (&o)[2]) {
        const float4 v = *reinterpret_cast<const float4 *>(p);
        o[0] = make_float2(v.x, v.y);
        o[1] = make_float2(v.z, v.w);
    }
    __device__ static uint4 bits(const float2 (&o)[2]) {
        return make_uint4(__float_as_uint(o[0].x), __float_as_uint(o[0].y), __float_as_uint(o[1].x),
                          __float_as_uint(o[1].y));
    }
};
template <> struct Chunk16<double2> {
    static constexpr int n = 1;
    __device__ static void load(const double2 *p, double2 (&o)[1]) { o[0] = *p; }
    __device__ static uint4 bits(const double2 (&o)[1]) {
        return make_uint4((unsigned)__double2loint(o[0].x), (unsigned)__double2hiint(o[0].x),
                          (unsigned)__double2loint(o[0].y), (unsigned)__double2hiint(o[0].y));
    }
};

// Staged form (the default).  CTA r of the cluster owns rows [r0, r0+nr) of
// z_j; its slab of Q_j (nr x 2nz', contiguous in global memory) is staged in
// shared memory by a bulk (TMA) copy issued a step ahead.  A warp owns RW rows;
// its 32 lanes split the K dimension, so every z_{j-1} element read from shared
// memory feeds RW rows x NBT columns of multiply-adds.  A butterfly reduce-
// scatter over the lanes leaves one finished complex per lane (or per lane
// pair/quad); the finished rows are pushed as 16-byte chunks to every CTA of
// the cluster, itself included, so one transaction-count mbarrier per step
// covers the whole z_j and no CTA-wide barrier is needed.
template <class T2, int NBT, int RW>
__global__ void __launch_bounds__(256) k_inner_sweep(const LayerDesc *__restrict__ layers,
                                                     const int *__restrict__ ids, const T2 *__restrict__ P,
                                                     const T2 *__restrict__ V, const T2 *__restrict__ H, T2 *X, int B,
                                                     int *err) {
    namespace cg = cooperative_groups;
    using Re = decltype(T2::x);
    using CK = Chunk16<T2>;
    constexpr int CPC = CK::n;           // complex values per 16-byte chunk
    constexpr int NBP = NBT + CPC;       // padded z row: 16-byte aligned, rows fall in different banks
    constexpr int NCH = NBT / CPC;       // chunks per row
    constexpr int VC = RW * NBT;         // complex outputs of a warp
    constexpr int SH = VC >= 32 ? 0 : (VC == 16 ? 1 : 2);  // lanes per output = 1 << SH
    constexpr int G = RW * NCH;          // chunks of a warp
    constexpr int LPC = 32 / G;          // lanes per chunk
    constexpr int PPL = 16 / LPC;        // pushes per lane (offsets 0..15 of the cluster)
    constexpr int QST = 2;               // Q slab stages
    static_assert(VC == 8 || VC == 16 || VC == 32, "warp output tile");
    static_assert(G >= 2 && G <= 32 && 32 % G == 0 && LPC <= 16, "chunk layout");
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ __align__(8) unsigned long long zbar[2], qbar[QST];
    cg::cluster_group cl = cg::this_cluster();
    const int R = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const int grp = blockIdx.x / R;
    const LayerDesc ld = layers[ids[blockIdx.y]];
    const int n2 = 2 * ld.nz, J = ld.C - 1;
    if (J <= 0) return;  // uniform over the cluster
    const int n0 = grp * NBT;
    const int rs = (n2 + R - 1) / R;
    const int r0 = min(n2, rank * rs), nr = min(n2, r0 + rs) - r0;
    T2 *zb0 = reinterpret_cast<T2 *>(smraw);
    T2 *zb1 = zb0 + n2 * NBP;
    T2 *qs = zb1 + n2 * NBP;  // QST slabs of rs x n2
    const long long slot = (long long)n2 * B;
    const T2 *h = H + ld.inner_off * (long long)B;
    T2 *x = X + ld.inner_off * (long long)B;
    const T2 *Pl = P + ld.P_off, *Vl = V + ld.V_off;
    const int tid = threadIdx.x, lane = tid & 31;
    const int mw = (tid >> 5) * RW;  // first row of this warp within the slab
    const bool wvalid = mw < nr;
    const int S = 2 * (J - 1);
    auto step_j = [&](int s) { return s < J - 1 ? s + 1 : J - 2 - (s - (J - 1)); };
    const unsigned qbytes = (unsigned)((long long)nr * n2 * sizeof(T2));
    auto issue_q = [&](int s) {  // one thread
        if (s >= S || qbytes == 0) return;
        const int b = s % QST;
        const unsigned mb = smem_u32(&qbar[b]);
        mbar_arrive_tx(mb, qbytes);
        const T2 *src = (s < J - 1 ? Pl : Vl) + (long long)step_j(s) * n2 * n2 + (long long)r0 * n2;
        bulk_g2s(smem_u32(qs + (long long)b * rs * n2), src, qbytes, mb);
    };
    if (tid == 0) {
        mbar_init(smem_u32(&zbar[0]), 1);
        mbar_init(smem_u32(&zbar[1]), 1);
        for (int i = 0; i < QST; i++) mbar_init(smem_u32(&qbar[i]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        issue_q(0);
    }
    // z_0 = h_0 into the first buffer; x_0's rows of this CTA start as h_0
    for (int e = tid; e < n2 * NBT; e += blockDim.x) {
        const int k = e / NBT, n = e % NBT;
        zb0[k * NBP + n] = (n0 + n < B) ? h[slot + (long long)k * B + n0 + n] : czero<T2>();
    }
    for (int e = tid; e < nr * NBT; e += blockDim.x) {
        const int m = r0 + e / NBT, n = e % NBT;
        if (n0 + n < B) x[slot + (long long)m * B + n0 + n] = h[slot + (long long)m * B + n0 + n];
    }
    // the finished output a lane holds after the reduction: row mw + r_me, column c_me
    const int f_me = lane >> SH;
    const int r_me = f_me / NBT, c_me = f_me % NBT;
    const bool own_valid = mw + r_me < nr && n0 + c_me < B;
    // the chunk a lane pushes (row gr, columns gc..gc+CPC-1) and its cluster offsets d0 + t * LPC
    const int g_me = lane % G, d0 = lane / G;
    const int gr = g_me / NCH, gc = CPC * (g_me % NCH);
    const bool push_valid = wvalid && mw + gr < nr;
    T2 bc = czero<T2>(), bn = czero<T2>();
    auto loadb = [&](int s, T2 &b) {
        if (s >= S) return;
        b = czero<T2>();
        if (own_valid)
            b = ((s < J - 1 ? h : x) + (long long)(step_j(s) + 1) * slot + (long long)(r0 + mw + r_me) * B + n0 +
                 c_me)[0];
    };
    loadb(0, bc);
    cl.sync();  // mbarriers initialised and z_0 written in every CTA
    const unsigned rx_bytes = (unsigned)((long long)n2 * NBT * sizeof(T2));
    unsigned zph = 0u, qph = 0u;
    bool dead = false;
    int q_next = 1;  // thread 0: next step whose Q slab it issues (step 0 was issued above)
    // Only warps that own rows take part in the steps.  Every such warp gates
    // every CTA of the cluster through its pushes, so no CTA runs more than one
    // step ahead of another and a phase of a barrier never receives bytes of a
    // later phase.  Warps (and whole CTAs, when 2nz' < R * rows-per-CTA) with no
    // rows receive nothing and wait for nothing; they go straight to the final
    // cluster barrier.
    for (int s = 0; s < S && wvalid; s++) {
        const int bo = (s & 1) ^ 1;  // z_s in buffer s&1, z_{s+1} into buffer bo
        const T2 *cur = bo ? zb0 : zb1;
        T2 *nxt = bo ? zb1 : zb0;
        if (tid == 0) {
            mbar_arrive_tx(smem_u32(&zbar[bo]), rx_bytes);
            issue_q(s + 1);  // its buffer was last read in step s-1, which every warp has left
            q_next = s + 2;
        }
        loadb(s + 1, bn);
        const int qb = s % QST;
        mbar_wait_bounded(smem_u32(&qbar[qb]), (qph >> qb) & 1u, false, dead, err);
        qph ^= 1u << qb;
        if (__any_sync(0xffffffffu, dead)) break;
        T2 acc[RW][NBT];
#pragma unroll
        for (int r = 0; r < RW; r++)
#pragma unroll
            for (int c = 0; c < NBT; c++) acc[r][c] = czero<T2>();
        if (wvalid) {
            const T2 *qrow = qs + (long long)qb * rs * n2 + (long long)mw * n2;
            for (int k = lane; k < n2; k += 32) {
                T2 q[RW];
#pragma unroll
                for (int r = 0; r < RW; r++) q[r] = (mw + r < nr) ? qrow[r * n2 + k] : czero<T2>();
                const T2 *zr = cur + k * NBP;
#pragma unroll
                for (int ch = 0; ch < NCH; ch++) {
                    T2 z[CPC];
                    CK::load(zr + ch * CPC, z);
#pragma unroll
                    for (int i = 0; i < CPC; i++)
#pragma unroll
                        for (int r = 0; r < RW; r++) cmac(acc[r][ch * CPC + i], q[r], z[i]);
                }
            }
        }
        // reduce-scatter of the warp's RW x NBT complex sums over its 32 lanes
        Re w[2 * VC];
#pragma unroll
        for (int r = 0; r < RW; r++)
#pragma unroll
            for (int c = 0; c < NBT; c++) {
                w[2 * (r * NBT + c)] = acc[r][c].x;
                w[2 * (r * NBT + c) + 1] = acc[r][c].y;
            }
#pragma unroll
        for (int o = 16, cnt = 2 * VC; cnt > 2; o >>= 1, cnt >>= 1) {
            const bool up = (lane & o) != 0;
            const int hf = cnt / 2;
#pragma unroll
            for (int j = 0; j < hf; j++) {
                const Re send = up ? w[j] : w[j + hf];
                const Re keep = up ? w[j + hf] : w[j];
                w[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
#pragma unroll
        for (int o = 1; o < (1 << SH); o <<= 1) {
            w[0] += __shfl_xor_sync(0xffffffffu, w[0], o);
            w[1] += __shfl_xor_sync(0xffffffffu, w[1], o);
        }
        T2 y;
        y.x = w[0] + bc.x;
        y.y = w[1] + bc.y;
        if (n0 + c_me >= B) y = czero<T2>();
        T2 pk[CPC];
#pragma unroll
        for (int i = 0; i < CPC; i++) {
            const int src = (gr * NBT + gc + i) << SH;
            pk[i].x = __shfl_sync(0xffffffffu, y.x, src);
            pk[i].y = __shfl_sync(0xffffffffu, y.y, src);
        }
        if (push_valid) {
            const int row = r0 + mw + gr;
            const unsigned a = smem_u32(nxt + row * NBP + gc);
            const unsigned mb = smem_u32(&zbar[bo]);
            const uint4 v = CK::bits(pk);
            if (d0 == 0) {
                T2 *outp = x + (long long)(step_j(s) + 1) * slot + (long long)row * B + n0 + gc;
#pragma unroll
                for (int i = 0; i < CPC; i++)
                    if (n0 + gc + i < B) outp[i] = pk[i];
            }
#pragma unroll
            for (int t = 0; t < PPL; t++) {
                const int d = d0 + t * LPC;
                if (d < R) {
                    int pr = rank + d;
                    if (pr >= R) pr -= R;
                    if (pr * rs < n2)  // CTAs without rows take no part
                        st_async16(cluster_map(a, pr), v, cluster_map(mb, pr));
                }
            }
        }
        // all of z_{s+1} (own rows included) has landed once the phase completes
        mbar_wait_bounded(smem_u32(&zbar[bo]), (zph >> bo) & 1u, true, dead, err);
        zph ^= 1u << bo;
        if (__any_sync(0xffffffffu, dead)) break;
        bc = bn;
    }
    // after a timeout: let this CTA's own bulk loads still in flight land (bounded)
    if (tid == 0 && dead) {
        for (int s = q_next - 1; s >= 0 && s > q_next - 1 - QST && s < S; s--) {
            const int b = s % QST;
            // the phase of buffer b that step s completes has parity (s / QST) & 1
            mbar_wait_bounded(smem_u32(&qbar[b]), (unsigned)((s / QST) & 1), false, dead, err);
        }
    }
    cl.sync();  // no CTA leaves while peers may still push into it
    if (__syncthreads_or(dead)) __nanosleep(20000);  // pushes a timed-out peer issued may still be landing
}

template <class T2, int NBT, int RW>
static bool inner_sweep_staged(const LayerDesc *d_layers, const int *ids, int nlayer, const T2 *P, const T2 *V,
                               const T2 *H, T2 *X, int B, int max_n2, int *err, cudaStream_t st, int Rfix = 0) {
    constexpr int CPC = 16 / (int)sizeof(T2);
    const int groups = (B + NBT - 1) / NBT;
    auto kern = k_inner_sweep<T2, NBT, RW>;
    HZ_CU(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    for (int R = Rfix ? Rfix : 16; R >= 2; R /= 2) {
        if (Rfix && R != Rfix) break;
        const int rs = (max_n2 + R - 1) / R;
        const int warps = (rs + RW - 1) / RW;
        if (warps > 8) return false;  // larger R would have been tried first
        if (!Rfix && RW == 4 && rs <= 16) continue;  // the RW = 2 form serves these slabs
        const size_t sm = (size_t)(2 * max_n2 * (NBT + CPC) + 2LL * rs * max_n2) * sizeof(T2);
        if (sm > 220 * 1024) continue;
        HZ_CU(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = R;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.blockDim = dim3(32 * warps, 1, 1);
        cfg.gridDim = dim3(R * groups, nlayer, 1);
        cfg.dynamicSmemBytes = sm;
        cfg.stream = st;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int ncl = 0;
        if (cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg) != cudaSuccess || ncl <= 0) {
            cudaGetLastError();
            continue;
        }
        HZ_CU(cudaLaunchKernelEx(&cfg, kern, d_layers, ids, P, V, H, X, B, err));
        return true;
    }
    return false;
}

// ---- launch-shape tuner of the staged sweep ----
// The candidates differ in right-hand sides per cluster (NBT), rows per warp
// (RW) and cluster size (R).  With tuning on, the first launch of each shape
// (precision, layers in flight, right-hand sides, largest 2nz') times every
// feasible candidate on the real data (the sweep is idempotent: x depends only
// on h, P and V) and keeps the fastest for the process; HZ_TUNE_CACHE names a
// JSON file that carries the choices across processes.
struct SweepCand {
    int nbt, rw, R;
};
static const SweepCand kSweepCands[] = {{8, 2, 16}, {16, 2, 16}, {8, 4, 16}, {8, 2, 8}, {16, 2, 8}, {8, 4, 8},
                                        {4, 4, 8},  {4, 8, 8},   {4, 2, 16}, {4, 4, 16}, {2, 4, 8},  {2, 8, 8},
                                        {2, 4, 16}};
constexpr int kNumSweepCands = (int)(sizeof(kSweepCands) / sizeof(kSweepCands[0]));

template <class T2>
static bool sweep_cand(int i, const LayerDesc *d_layers, const int *ids, int nlayer, const T2 *P, const T2 *V,
                       const T2 *H, T2 *X, int B, int max_n2, int *err, cudaStream_t st) {
    const SweepCand &k = kSweepCands[i];
    if (k.nbt == 8 && k.rw == 2)
        return inner_sweep_staged<T2, 8, 2>(d_layers, ids, nlayer, P, V, H, X, B, max_n2, err, st, k.R);
    if (k.nbt == 16 && k.rw == 2)
        return inner_sweep_staged<T2, 16, 2>(d_layers, ids, nlayer, P, V, H, X, B, max_n2, err, st, k.R);
    if (k.nbt == 8 && k.rw == 4)
        return inner_sweep_staged<T2, 8, 4>(d_layers, ids, nlayer, P, V, H, X, B, max_n2, err, st, k.R);
    if (k.nbt == 4 && k.rw == 2)
        return inner_sweep_staged<T2, 4, 2>(d_layers, ids, nlayer, P, V, H, X, B, max_n2, err, st, k.R);
    if (k.nbt == 4 && k.rw == 4)
        return inner_sweep_staged<T2, 4, 4>(d_layers, ids, nlayer, P, V, H, X, B, max_n2, err, st, k.R);
    if (k.nbt == 4 && k.rw == 8)
        return inner_sweep_staged<T2, 4, 8>(d_layers, ids, nlayer, P, V, H, X, B, max_n2, err, st, k.R);
    if (k.nbt == 2 && k.rw == 4)
        return inner_sweep_staged<T2, 2, 4>(d_layers, ids, nlayer, P, V, H, X, B, max_n2, err, st, k.R);
    if (k.nbt == 2 && k.rw == 8)
        return inner_sweep_staged<T2, 2, 8>(d_layers, ids, nlayer, P, V, H, X, B, max_n2, err, st, k.R);
    return false;
}

struct TuneTable {
    std::mutex mu;
    std::map<std::string, int> best;
    bool loaded = false;
    static std::string path() {
        const char *p = std::getenv("HZ_TUNE_CACHE");
        return p ? std::string(p) : std::string();
    }
    void load_locked() {  // {"key": value, ...}; anything unreadable is ignored
        loaded = true;
        const std::string p = path();
        if (p.empty()) return;
        std::ifstream f(p);
        if (!f) return;
        std::stringstream ss;
        ss << f.rdbuf();
        const std::string t = ss.str();
        size_t i = 0;
        while ((i = t.find('"', i)) != std::string::npos) {
            const size_t j = t.find('"', i + 1);
            if (j == std::string::npos) break;
            const std::string key = t.substr(i + 1, j - i - 1);
            const size_t c = t.find(':', j);
            if (c == std::string::npos) break;
            best[key] = std::atoi(t.c_str() + c + 1);
            i = t.find_first_of(",}", c);
            if (i == std::string::npos) break;
        }
    }
    void save_locked() {
        const std::string p = path();
        if (p.empty()) return;
        std::ofstream f(p);
        if (!f) return;
        f << "{";
        bool first = true;
        for (auto &kv : best) {
            f << (first ? "" : ",") << "\n  \"" << kv.first << "\": " << kv.second;
            first = false;
        }
        f << "\n}\n";
    }
};
static TuneTable &tune_table() {
    static TuneTable t;
    return t;
}

template <class T2>
static int tune_sweep(const std::string &key, const LayerDesc *d_layers, const int *ids, int nlayer, const T2 *P,
                      const T2 *V, const T2 *H, T2 *X, int B, int max_n2, int *err, cudaStream_t st) {
    cudaEvent_t e0, e1;
    HZ_CU(cudaEventCreate(&e0));
    HZ_CU(cudaEventCreate(&e1));
    int best = -1;
    float best_ms = 0.f;
    for (int i = 0; i < kNumSweepCands; i++) {
        float ms = 1e30f;
        bool ok = true;
        for (int rep = 0; rep < 3 && ok; rep++) {
            HZ_CU(cudaEventRecord(e0, st));
            try {
                ok = sweep_cand<T2>(i, d_layers, ids, nlayer, P, V, H, X, B, max_n2, err, st);
            } catch (const CudaError &) {
                cudaGetLastError();
                ok = false;
            }
            HZ_CU(cudaEventRecord(e1, st));
            HZ_CU(cudaEventSynchronize(e1));
            float t = 0.f;
            HZ_CU(cudaEventElapsedTime(&t, e0, e1));
            if (ok) ms = std::min(ms, t);
        }
        if (ok && (best < 0 || ms < best_ms)) {
            best = i;
            best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    TuneTable &tt = tune_table();
    std::lock_guard<std::mutex> lk(tt.mu);
    tt.best[key] = best;
    tt.save_locked();
    return best;
}

template <class T2>
void launch_inner_sweep(const LayerDesc *d_layers, const int *ids, int nlayer, const T2 *P, const T2 *V,
                        const T2 *H, T2 *X, int B, int max_n2, int *err, cudaStream_t st, int *nl, bool tune) {
    if (nlayer <= 0 || B <= 0) return;
    bool ok = false;
    if (tune) {
        int dev = 0;
        cudaGetDevice(&dev);
        char key[160];
        snprintf(key, sizeof key, "sweep es=%d layers=%d rhs=%d n2=%d dev=%d", (int)sizeof(T2), nlayer, B, max_n2, dev);
        int choice = -2;
        {
            TuneTable &tt = tune_table();
            std::lock_guard<std::mutex> lk(tt.mu);
            if (!tt.loaded) tt.load_locked();
            auto it = tt.best.find(key);
            if (it != tt.best.end()) choice = it->second;
        }
        if (choice == -2) choice = tune_sweep<T2>(key, d_layers, ids, nlayer, P, V, H, X, B, max_n2, err, st);
        if (choice >= 0 && choice < kNumSweepCands)
            ok = sweep_cand<T2>(choice, d_layers, ids, nlayer, P, V, H, X, B, max_n2, err, st);
    }
    // default rule (what the tuner picks on the 1024 x 1024 and the multi-frequency
    // 512 x 512 shapes): 4-column tiles in 8-CTA clusters with 4 rows per warp, unless
    // that leaves SMs idle (a single layer with few right-hand sides): then 2-column
    // tiles (8-CTA clusters in FP32, 16-CTA clusters in FP64).  Interface blocks whose
    // row slabs do not fit 8 CTAs (2nz' = 320 on the 2000 x 4000 shape): a single layer
    // takes 4-column tiles in 16-CTA clusters, several layers 8-column tiles (the
    // tuner's choices there).
    static int n_sm = 0;
    if (n_sm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n_sm <= 0) n_sm = 152;
    }
    const bool narrow = (long long)((B + 7) / 8) * nlayer * 16 <= 608;
    if (!ok && (long long)((B + 3) / 4) * nlayer * 8 < n_sm)
        ok = inner_sweep_staged<T2, 2, 4>(d_layers, ids, nlayer, P, V, H, X, B, max_n2, err, st, sizeof(T2) == 8 ? 8 : 16);
    if (!ok) ok = inner_sweep_staged<T2, 4, 4>(d_layers, ids, nlayer, P, V, H, X, B, max_n2, err, st, 8);
    if (!ok && nlayer == 1)
        ok = inner_sweep_staged<T2, 8, 4>(d_layers, ids, nlayer, P, V, H, X, B, max_n2, err, st, 8);
    if (!ok && nlayer == 1) ok = inner_sweep_staged<T2, 4, 4>(d_layers, ids, nlayer, P, V, H, X, B, max_n2, err, st, 16);
    if (!ok) ok = inner_sweep_staged<T2, 8, 2>(d_layers, ids, nlayer, P, V, H, X, B, max_n2, err, st);
    if (!ok) ok = inner_sweep_staged<T2, 8, 4>(d_layers, ids, nlayer, P, V, H, X, B, max_n2, err, st);
    if (!ok) {
        if (narrow)
            ok = inner_sweep_regq<T2, 8>(d_layers, ids, nlayer, P, V, H, X, B, max_n2, err, st);
        else
            ok = inner_sweep_regq<T2, 16>(d_layers, ids, nlayer, P, V, H, X, B, max_n2, err, st) ||
                 inner_sweep_regq<T2, 8>(d_layers, ids, nlayer, P, V, H, X, B, max_n2, err, st);
    }
    if (!ok) throw HzError(HZ_ENOMEM, "inner sweep: interface blocks too large for shared memory");
    if (nl) (*nl)++;
}
template void launch_inner_sweep<double2>(const LayerDesc *, const int *, int, const double2 *, const double2 *,
                                          const double2 *, double2 *, int, int, int *, cudaStream_t, int *, bool);
template void launch_inner_sweep<float2>(const LayerDesc *, const int *, int, const float2 *, const float2 *,
                                         const float2 *, float2 *, int, int, int *, cudaStream_t, int *, bool);

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
    const int ldw = cd.ldw;
    const long long nn = (long long)nx * ldw;
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
                a = a - (c1 * Wp[(long long)i * ldw + k]) * c2;
            }
            S[(long long)i * ldw + k] = a;
        }
        __syncthreads();
        int r = gj_inverse(S, nx, ldw, rowk, colk, perm, redv, redi);
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


// ================================================= persistent narrow sweep ===
// A whole Gauss-Seidel sweep (every step's [P2, P1], Λ and P3 lists of §8e, in
// order) as one cooperative launch: the CTAs stay resident and take the work
// units of a phase (problem, 32-row tile, K slice) in turn, and the phases are
// separated by a grid barrier.  The barrier is a counter that every CTA raises
// once per phase and polls with acquire loads; the wait is bounded by the
// context's wait limit, after which the CTA sets the error word and leaves (the
// others see the error word and leave too), so a failed barrier ends the launch
// with HZ_ETIMEOUT instead of hanging.
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <int NB>
__global__ void __launch_bounds__(NW_WPC * 32) k_narrow_sweep(const NwPhase *__restrict__ ph, int nph, float2 *ws,
                                                              int *cnt, unsigned *bar, int *err) {
    __shared__ GemmProb<float2> P;
    __shared__ int last, dead;
    extern __shared__ __align__(16) unsigned char nsm[];
    for (int f = 0; f < nph; f++) {
        const NwPhase Q = ph[f];
        const int per = Q.max_tiles * Q.split, units = Q.n * per;
        for (int u = blockIdx.x; u < units; u += gridDim.x) {
            const int pr = u / per, rem = u - pr * per, tile = rem / Q.split, sp = rem - tile * Q.split;
            narrow_unit<NB, true>(Q.d + pr, tile, sp, Q.split, ws, cnt, (long long)pr * Q.max_tiles + tile, P, last,
                                  nsm);
        }
        if (f + 1 == nph) break;
        __syncthreads();  // this CTA's stores of the phase are issued
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(bar, 1u);
            const unsigned target = (unsigned)(f + 1) * gridDim.x;
            const unsigned long long lim = wait_limit_ns(err);
            unsigned long long t0 = 0;
            int d = 0;
            for (unsigned it = 0;; it++) {
                if (ld_acquire_u32(bar) >= target) break;
                if ((it & 63u) == 63u) {
                    if (*reinterpret_cast<volatile int *>(err)) {  // another CTA gave up
                        d = 1;
                        break;
                    }
                    const unsigned long long t = global_ns();
                    if (t0 == 0) {
                        t0 = t;
                    } else if (t - t0 > lim) {
                        atomicExch(err, 1);
                        d = 1;
                        break;
                    }
                }
                __nanosleep(64);
            }
            __threadfence();
            dead = d;
        }
        __syncthreads();
        if (dead) return;
    }
}

int narrow_sweep_grid() {
    static int g = -1;
    if (g < 0) {
        int dev = 0, sms = 0, per = 0, coop = 0;
        HZ_CU(cudaGetDevice(&dev));
        HZ_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        HZ_CU(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
        const size_t sm = nw_smem<NW_NB>();
        HZ_CU(cudaFuncSetAttribute(k_narrow_sweep<NW_NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        HZ_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_narrow_sweep<NW_NB>, NW_WPC * 32, sm));
        g = coop ? std::min(per, NW_CTAS_PER_SM) * sms : 0;
    }
    return g;
}

void launch_narrow_sweep(const NwPhase *d_ph, int nph, float2 *ws, int *cnt, unsigned *bar, int *err, int grid,
                         cudaStream_t st, int *nl) {
    if (nph <= 0) return;
    if (grid <= 0 || grid > narrow_sweep_grid()) throw HzError(HZ_EINVAL, "persistent sweep: grid not co-resident");
    HZ_CU(cudaMemsetAsync(bar, 0, sizeof(unsigned), st));
    void *args[] = {(void *)&d_ph, (void *)&nph, (void *)&ws, (void *)&cnt, (void *)&bar, (void *)&err};
    HZ_CU(cudaLaunchCooperativeKernel((const void *)k_narrow_sweep<NW_NB>, dim3(grid), dim3(NW_WPC * 32), args,
                                      nw_smem<NW_NB>(), st));
    if (nl) (*nl)++;
}

}  // namespace hz
