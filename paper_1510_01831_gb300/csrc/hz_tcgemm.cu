// Tensor-core form of the batched segmented complex GEMM (mixed precision,
// sm_103a tcgen05): the F, E and S products of the layer applications
// (eq. (factorization); Section 4.2) and the h_j = W_j g_j products of the
// inner solves, Y (+)= alpha (A X + A2 X2) with A, A2 FP32 complex operators
// and X, X2 row-segmented right-hand-side panels (the problem descriptor of
// the SIMT kernel).
//
// Every complex product runs as real products with the 3xTF32 split
// X Y ~ Xh Yh + Xh Yl + Xl Yh (Xh = X rounded to TF32, Xl = X - Xh rounded to
// TF32).  The real part takes Ar Xr + Ai (-Xi), the imaginary part Ar Xi + Ai Xr,
// so that one accumulator serves each (main Xh Yh terms and small cross terms
// apart): four accumulators of 64 columns per K chunk, filled by 4 MMAs per K
// step of 8 -- Ar_h and Ai_h against the 256-row operands [Xr_h; Xi_h; Xr_l;
// Xi_l] and [-Xi_h; Xr_h; -Xi_l; Xr_l] (N = 256), Ar_l and Ai_l against their
// first 128 rows (N = 128, cross columns only).
//
// The operators are constant: each distinct operator block is split once
// (tc_split_operator) into TF32 planes Ar_h, Ar_l, Ai_h, Ai_l laid out per
// (128-row tile, 16-column chunk) in the no-swizzle K-major canonical layout
// of the MMA operand, only the tile's rows rounded up to 8 stored, so that one
// chunk of A is one contiguous bulk copy.
//
// CTA = one 128 x 64 output tile (MMA M = 128 rows of A, N = 64 right-hand
// sides) over a range of K chunks of 16 (split-K across CTAs when a launch has
// few tiles).  Roles:
//   - warps 4-7 (converters) copy the X chunk (16 x 64) from global memory with
//     asynchronous copies, two chunks ahead, into raw stages (each thread
//     copies exactly what it later converts), split it into the TF32 planes of
//     the two 256-row operands and store them in the canonical layout, into 2
//     X stages;
//   - warps 0-3 (thread = output row = TMEM lane) drain each chunk's
//     accumulator set with tcgen05.ld and add it into FP32 registers, so that
//     no accumulator in tensor memory takes more than 4 additions (the tensor
//     core's accumulation truncates; register sums round to nearest), then
//     store the tile through shared memory with row-contiguous writes;
//   - warp 0 also drives the tensor cores: once chunk i's products have
//     completed it bulk-copies the A chunk i + 4 into the freed stage of a
//     4-stage A ring, and after draining chunk i it issues chunk i + 2 (2 K
//     steps of 8 x 4 products) into the freed accumulator set while chunk
//     i + 1 runs.
// Split-K partial tiles go to a workspace; the last CTA of a tile to arrive
// adds them in split order (deterministic) and writes the output.
// Every wait is bounded (1 s): a timeout sets the error word, the CTA leaves
// its loops, lets its bulk copies land, skips its output and frees its tensor
// memory.
#include <map>
#include <tuple>

#include "hz_ctx.cuh"
#include "hz_tc.cuh"

namespace hz {

namespace {

constexpr int GT_THREADS = 256;                      // 8 warps (see the file header)
constexpr int GT_D = 2;                              // X chunks in flight (asynchronous copies)
constexpr int GT_RAW = GT_D + 1;                     // raw X stages
constexpr int GT_XS = 2;                             // X plane stages
constexpr int GT_AS = 4;                             // A stages
constexpr int GT_RAWB = GT_KC * GT_N * 8;            // bytes per raw X stage
constexpr int GT_APL = GT_M * GT_KC * 4;             // bytes per A plane of a full chunk
constexpr int GT_XPL = GT_N * GT_KC * 4;             // bytes per X plane of a chunk
constexpr int GT_ASTG = 4 * GT_APL;                  // bytes per A stage
constexpr int GT_XSTG = 8 * GT_XPL;                  // bytes per X stage
constexpr int GT_SMEM = GT_AS * GT_ASTG + GT_XS * GT_XSTG + GT_RAW * GT_RAWB;  // dynamic shared memory
constexpr int GT_SR = GT_N + 2;  // output staging row (float2): 16-byte rows, conflict-free 16-byte stores
static_assert(GT_M * GT_SR * 8 <= GT_AS * GT_ASTG, "output staging fits the A ring");

__device__ __forceinline__ void split_tf32(float x, float &h, float &l) {
    h = tf32_rna(x);
    l = tf32_rna(x - h);
}

__device__ __forceinline__ void cp_async8(unsigned dst, const void *src, unsigned bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Converter thread (warp cw of the four, lane): its share of an X chunk is the
// entries of K rows 4 cw..4 cw+3, columns lane and lane + 32.  It copies
// exactly the bytes it later converts, so the copies need no barrier between
// threads.  Entries outside the operand are zero-filled by the copies.
__device__ __forceinline__ void gt_copy_x(const GemmProb<float2> &P, int q, int n1, int K1, int K2, int n0, int N,
                                          int cw, int lane, unsigned raw) {
    const bool p2 = q >= n1;
    const int k0 = (p2 ? q - n1 : q) * GT_KC, Kp = p2 ? K2 : K1;
    const int xseg = p2 ? P.xseg2 : P.xseg;
    const long long ldx = p2 ? P.ldx2 : P.ldx;
    const float2 *any = p2 ? P.X2[0] : P.X[0];  // a valid address for zero-byte copies
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int kx = 4 * cw + i, gk = k0 + kx;
        const float2 *xr = any;
        const bool kok = gk < Kp;
        if (kok) {
            const int sg = gk / xseg;
            xr = (p2 ? P.X2[sg] : P.X[sg]) + (long long)(gk - sg * xseg) * ldx + n0;
        }
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int n = lane + 32 * h;
            const bool ok = kok && n0 + n < N;
            cp_async8(raw + kx * (GT_N * 8) + n * 8, ok ? (const void *)(xr + n) : (const void *)any, ok ? 8u : 0u);
        }
    }
}

// converter thread: split its landed share of an X chunk into the planes of an
// X stage: two B operands of 256 rows (4 planes of 64 right-hand sides each),
// [Xr_h; Xi_h; Xr_l; Xi_l] and [-Xi_h; Xr_h; -Xi_l; Xr_l]
__device__ __forceinline__ void gt_convert_x(const unsigned char *raw, unsigned char *sx, int cw, int lane) {
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int n = lane + 32 * h;
        float2 x[4];
#pragma unroll
        for (int i = 0; i < 4; i++) x[i] = *reinterpret_cast<const float2 *>(raw + (4 * cw + i) * (GT_N * 8) + n * 8);
        float4 rh, rl, ih, il;
        split_tf32(x[0].x, rh.x, rl.x);
        split_tf32(x[1].x, rh.y, rl.y);
        split_tf32(x[2].x, rh.z, rl.z);
        split_tf32(x[3].x, rh.w, rl.w);
        split_tf32(x[0].y, ih.x, il.x);
        split_tf32(x[1].y, ih.y, il.y);
        split_tf32(x[2].y, ih.z, il.z);
        split_tf32(x[3].y, ih.w, il.w);
        const unsigned o = canon(n, 4 * cw, GT_KC);
        *reinterpret_cast<float4 *>(sx + 0 * GT_XPL + o) = rh;
        *reinterpret_cast<float4 *>(sx + 1 * GT_XPL + o) = ih;
        *reinterpret_cast<float4 *>(sx + 2 * GT_XPL + o) = rl;
        *reinterpret_cast<float4 *>(sx + 3 * GT_XPL + o) = il;
        *reinterpret_cast<float4 *>(sx + 4 * GT_XPL + o) = make_float4(-ih.x, -ih.y, -ih.z, -ih.w);
        *reinterpret_cast<float4 *>(sx + 5 * GT_XPL + o) = rh;
        *reinterpret_cast<float4 *>(sx + 6 * GT_XPL + o) = make_float4(-il.x, -il.y, -il.z, -il.w);
        *reinterpret_cast<float4 *>(sx + 7 * GT_XPL + o) = rl;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
}

// rows of tile mt stored in the split copy (the tile's rows rounded up to 8)
__host__ __device__ __forceinline__ int atc_rows(int M, int mt) {
    const int r = min(GT_M, M - GT_M * mt);
    return 8 * ((r + 7) / 8);
}

// Split one operator block A (M x K, row-major, leading dimension lda) into
// the per-(tile, chunk) TF32 planes described in the file header:
// block (mt, c) at 128 * 64 * nc * mt + c * rows * 64 floats, planes of rows x 16.
__global__ void k_build_atc(const float2 *__restrict__ A, long long lda, int M, int K, float *dst) {
    const int nc = (K + GT_KC - 1) / GT_KC, nt = (M + GT_M - 1) / GT_M;
    const long long rows_total = (long long)GT_M * (nt - 1) + atc_rows(M, nt - 1);
    const long long n = rows_total * nc * GT_KC;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int kk = (int)(e % (nc * GT_KC));
        const int r = (int)(e / (nc * GT_KC));
        const int mt = r / GT_M, rr = r % GT_M, rows = atc_rows(M, mt);
        const int c = kk / GT_KC, k = kk % GT_KC;
        const float2 v = (r < M && kk < K) ? A[(long long)r * lda + kk] : make_float2(0.f, 0.f);
        float rh, rl, ih, il;
        split_tf32(v.x, rh, rl);
        split_tf32(v.y, ih, il);
        float *blk = dst + (long long)GT_M * 64 * nc * mt + (long long)c * rows * 64;
        const int off = (int)(canon(rr, k, GT_KC) / 4), pl = rows * GT_KC;
        blk[off] = rh;
        blk[pl + off] = rl;
        blk[2 * pl + off] = ih;
        blk[3 * pl + off] = il;
    }
}

__global__ void __launch_bounds__(GT_THREADS, 1)
    k_gemm_tc(const GemmProb<float2> *__restrict__ probs, int S, float2 *ws, int *cnt, int max_tiles, int *err) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    __shared__ GemmProb<float2> P;
    __shared__ __align__(8) unsigned long long afull[GT_AS], xfull[GT_XS], xempty[GT_XS], accfull[2], accempty[2];
    __shared__ unsigned tmem_slot;
    __shared__ volatile int s_dead;
    __shared__ int s_last, s_acopies, s_await;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) P = probs[blockIdx.y];
    __syncthreads();
    const int M = P.M, N = P.N;
    const int tilesM = (M + GT_M - 1) / GT_M, tilesN = (N + GT_N - 1) / GT_N;
    const int tile = blockIdx.x / S, sp = blockIdx.x % S;
    if (tile >= tilesM * tilesN) return;  // uniform over the CTA
    const int mt = tile % tilesM, m0 = mt * GT_M, n0 = (tile / tilesM) * GT_N;
    const int rows = atc_rows(M, mt);  // rows of this tile's A chunks
    // K chunks of 16 over the two passes laid end to end; split sp takes [qb, qe)
    const int K1 = max(P.K, 0), K2 = max(P.K2, 0);
    const int n1 = (K1 + GT_KC - 1) / GT_KC, n2 = (K2 + GT_KC - 1) / GT_KC, nch = n1 + n2;
    const int per = (nch + S - 1) / S;
    const int qb = min(nch, sp * per), qe = min(nch, qb + per), nq = qe - qb;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_slot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < GT_AS; i++) mb_init(su32(&afull[i]), 1);  // expect_tx arrival + copy bytes
        for (int i = 0; i < GT_XS; i++) {
            mb_init(su32(&xfull[i]), 128);  // the 128 converter threads
            mb_init(su32(&xempty[i]), 1);   // tcgen05.commit
        }
        for (int i = 0; i < 2; i++) {
            mb_init(su32(&accfull[i]), 1);     // tcgen05.commit
            mb_init(su32(&accempty[i]), 128);  // the 128 drain threads
        }
        s_dead = 0;
        s_acopies = 0;
        s_await = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = tmem_slot;
    unsigned char *aring = smraw, *xring = smraw + GT_AS * GT_ASTG, *rawb = xring + GT_XS * GT_XSTG;
    bool dead = false;

    if (warp >= 4) {
        // ---------------------------------------------------------- converters (X)
        const int cw = warp - 4;
        const unsigned raw0 = su32(rawb);
#pragma unroll
        for (int j = 0; j < GT_D; j++) {  // prologue: the first GT_D chunks in flight (one group each)
            if (j < nq) gt_copy_x(P, qb + j, n1, K1, K2, n0, N, cw, lane, raw0 + (j % GT_RAW) * GT_RAWB);
            cp_commit();
        }
        for (int i = 0; i < nq; i++) {
            const int st = i % GT_XS;
            // raw stage (i + D) % RAW last held chunk i - 1, which this thread has converted
            if (i + GT_D < nq)
                gt_copy_x(P, qb + i + GT_D, n1, K1, K2, n0, N, cw, lane, raw0 + ((i + GT_D) % GT_RAW) * GT_RAWB);
            cp_commit();
            cp_wait<GT_D>();  // this thread's copies of chunk i have landed
            // waits are taken by all lanes of the warp together
            const bool ok = i < GT_XS || mb_wait(su32(&xempty[st]), (unsigned)(((i / GT_XS) - 1) & 1), dead, err);
            if (__any_sync(0xffffffffu, !ok || s_dead)) {
                s_dead = 1;
                break;
            }
            gt_convert_x(rawb + (i % GT_RAW) * GT_RAWB, xring + st * GT_XSTG, cw, lane);
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&xfull[st])) : "memory");
        }
        cp_wait<0>();  // no copy in flight past this point
    } else {
        // ---------------------------------------------------------- drain (+ warp 0: A copies, MMA issue)
        float sr[GT_N], si[GT_N];  // the tile row's sums
#pragma unroll
        for (int j = 0; j < GT_N; j++) sr[j] = si[j] = 0.f;
        const unsigned ta = tmem + ((unsigned)(32 * warp) << 16);
        // D f32, A and B tf32, both K-major, M = 128, N = 256 (main products) or 128 (cross)
        const unsigned idesc_base = (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(GT_M >> 4) << 24);
        const unsigned idesc256 = idesc_base | ((unsigned)(4 * GT_N >> 3) << 17);
        const unsigned idesc128 = idesc_base | ((unsigned)(2 * GT_N >> 3) << 17);
        const unsigned abytes = (unsigned)rows * 4 * GT_KC * 4;  // one A chunk: 4 planes of rows x 16
        // lane 0 of warp 0: bulk-copy A chunk j into stage j % 4 (the stage's previous
        // chunk, j - 4, has completed its products)
        auto copy_a = [&](int j) {
            const int q = qb + j;
            const bool p2 = q >= n1;
            const float *src = p2 ? P.A2tc + (long long)GT_M * 64 * n2 * mt + (long long)(q - n1) * rows * 64
                                  : P.Atc + (long long)GT_M * 64 * n1 * mt + (long long)q * rows * 64;
            const int s = j % GT_AS;
            mb_expect(su32(&afull[s]), abytes);
            bulk_g2s(su32(aring + s * GT_ASTG), src, abytes, su32(&afull[s]));
            s_acopies = j + 1;
        };
        // warp 0 issues chunk j into accumulator set j & 1 once its A and X stages are
        // full (all lanes wait together; lane 0 issues)
        auto issue = [&](int j) {
            const int xs = j % GT_XS, as = j % GT_AS;
            bool okw = mb_wait(su32(&afull[as]), (unsigned)((j / GT_AS) & 1), dead, err);
            okw = okw && mb_wait(su32(&xfull[xs]), (unsigned)((j / GT_XS) & 1), dead, err);
            if (__any_sync(0xffffffffu, !okw)) return false;  // warp-uniform
            if (lane == 0) {
                s_await = j + 1;
                tc_fence_after();
                const unsigned sa = su32(aring + as * GT_ASTG), sx = su32(xring + xs * GT_XSTG);
                const unsigned d = tmem + 256u * (j & 1);  // re main, im main, re cross, im cross: +0, +64, +128, +192
                const unsigned apl = (unsigned)rows * GT_KC * 4;  // bytes per A plane of this tile's chunks
#pragma unroll
                for (int t = 0; t < GT_KC / 8; t++) {
                    auto A = [&](int p) { return sdesc(sa + p * apl + 256 * t, 128, (GT_KC / 4) * 128); };
                    const unsigned long long B1 = sdesc(sx + 256 * t, 128, (GT_KC / 4) * 128);               // [Xr_h; Xi_h; Xr_l; Xi_l]
                    const unsigned long long B2 = sdesc(sx + 4 * GT_XPL + 256 * t, 128, (GT_KC / 4) * 128);  // [-Xi_h; Xr_h; -Xi_l; Xr_l]
                    const unsigned f = t > 0 ? 1u : 0u;  // each chunk starts its set afresh
                    umma_tf32(d + 0, A(0), B1, idesc256, f);     // Ar_h: re, im main; Ar_h Xr_l, Ar_h Xi_l cross
                    umma_tf32(d + 0, A(2), B2, idesc256, 1u);    // Ai_h: -Ai_h Xi_h, Ai_h Xr_h; -Ai_h Xi_l, Ai_h Xr_l
                    umma_tf32(d + 128, A(1), B1, idesc128, 1u);  // Ar_l Xr_h, Ar_l Xi_h (cross)
                    umma_tf32(d + 128, A(3), B2, idesc128, 1u);  // -Ai_l Xi_h, Ai_l Xr_h (cross)
                }
                umma_commit(su32(&xempty[xs]));      // the converters may refill this X stage
                umma_commit(su32(&accfull[j & 1]));  // the drain warps may read this set
            }
            __syncwarp();
            return true;
        };
        bool ok = true;
        if (warp == 0) {
            if (lane == 0)
                for (int j = 0; j < GT_AS && j < nq; j++) copy_a(j);
            __syncwarp();
            for (int j = 0; j < 2 && j < nq && ok; j++) ok = issue(j);  // both sets start free
        }
        if (!ok) dead = true;
        for (int i = 0; i < nq && !dead; i++) {
            const int set = i & 1;
            if (!mb_wait(su32(&accfull[set]), (unsigned)((i / 2) & 1), dead, err)) s_dead = 1;
            if (__any_sync(0xffffffffu, dead || s_dead)) {  // warp-uniform: the loads below are .sync.aligned
                dead = true;
                break;
            }
            tc_fence_after();
            if (warp == 0 && lane == 0 && i + GT_AS < nq) copy_a(i + GT_AS);  // chunk i's products are done
#pragma unroll
            for (int pc = 0; pc < GT_N / 8; pc++) {
                float rm[8], im[8], rx[8], ix[8];
                const unsigned c = ta + 256u * set + 8u * pc;
                tmem_ld8(c, rm);
                tmem_ld8(c + 64, im);
                tmem_ld8(c + 128, rx);
                tmem_ld8(c + 192, ix);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 8; j++) {
                    sr[8 * pc + j] += rm[j] + rx[j];
                    si[8 * pc + j] += im[j] + ix[j];
                }
            }
            tc_fence_before();
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&accempty[set])) : "memory");
            if (warp == 0 && i + 2 < nq) {
                // set i & 1 is free once all four drain warps have read chunk i
                ok = mb_wait(su32(&accempty[set]), (unsigned)((i / 2) & 1), dead, err);
                if (__any_sync(0xffffffffu, !ok) || !issue(i + 2)) {
                    dead = true;
                    break;
                }
            }
        }
        if (dead) {
            s_dead = 1;
        } else {
            // stage the row in shared memory: the A ring is free once the last product has
            // completed
            float4 *stg4 = reinterpret_cast<float4 *>(smraw) + tid * (GT_SR / 2);  // row tid of [128][GT_SR] float2
#pragma unroll
            for (int j = 0; j < GT_N; j += 2) stg4[j / 2] = make_float4(sr[j], si[j], sr[j + 1], si[j + 1]);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (s_dead) {
        // after a timeout: let the A copies issued for this CTA land, and products still in
        // flight finish, before the shared and tensor memory are released
        if (tid == 0)
            for (int j = s_await; j < s_acopies; j++)
                mb_wait(su32(&afull[j % GT_AS]), (unsigned)((j / GT_AS) & 1), dead, err);
        __nanosleep(20000);
    }
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    if (s_dead || warp >= 4) return;  // (warps 4-7 hold no tensor memory)

    // ------------------------------------------------------------ output
    // (warps 0-3 only)
    float2 *stg = reinterpret_cast<float2 *>(smraw);  // [128][GT_SR], written by the drain loop
    const float al = P.alpha;
    if (S > 1) {
        // split-K: store this split's partial tile; the last split of the tile to arrive
        // adds the partials in split order and writes the output.  Float4 f of a tile
        // (f = tid + 128 k) holds complex columns 2 (f % 32), +1 of row f / 32.
        constexpr int F4 = GT_M * GT_N / 2;  // float4 per tile
        const long long slot = (long long)blockIdx.y * max_tiles + tile;
        float4 *wst = reinterpret_cast<float4 *>(ws) + slot * S * F4;
        const float4 *stg4 = reinterpret_cast<const float4 *>(smraw);
#pragma unroll 8
        for (int k = 0; k < F4 / 128; k++) {
            const int f = tid + 128 * k;
            wst[sp * F4 + f] = stg4[(f >> 5) * (GT_SR / 2) + (f & 31)];
        }
        __threadfence();
        asm volatile("bar.sync 1, 128;" ::: "memory");
        if (tid == 0) s_last = atomicAdd(&cnt[slot], 1) == S - 1;
        asm volatile("bar.sync 1, 128;" ::: "memory");
        if (!s_last) return;
        __threadfence();
        float4 *stw = reinterpret_cast<float4 *>(smraw);
        for (int kb = 0; kb < F4 / 128; kb += 4) {
            float4 acc[4];
#pragma unroll
            for (int u = 0; u < 4; u++) acc[u] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
            for (int q = 0; q < S; q++) {  // split order: deterministic
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const float4 w = __ldcg(wst + q * F4 + tid + 128 * (kb + u));
                    acc[u].x += w.x;
                    acc[u].y += w.y;
                    acc[u].z += w.z;
                    acc[u].w += w.w;
                }
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int f = tid + 128 * (kb + u);
                stw[(f >> 5) * (GT_SR / 2) + (f & 31)] = acc[u];
            }
        }
        if (tid == 0) cnt[slot] = 0;
        asm volatile("bar.sync 1, 128;" ::: "memory");
    }
#pragma unroll 2
    for (int rr = 32 * warp; rr < 32 * warp + 32; rr++) {
        const int m = m0 + rr;
        if (m >= M) break;
        const int sg = m / P.yseg;
        float2 *row = P.Y[sg] + (long long)(m - sg * P.yseg) * P.ldy + n0;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int n = lane + 32 * h;
            if (n0 + n >= N) continue;
            float2 v = stg[rr * GT_SR + n];
            v.x *= al;
            v.y *= al;
            if (P.beta) {
                const float2 y = row[n];
                v.x += y.x;
                v.y += y.y;
            }
            row[n] = v;
        }
    }
}

}  // namespace

long long atc_floats(int M, int K) {
    if (M <= 0 || K <= 0) return 0;
    const int nc = (K + GT_KC - 1) / GT_KC, nt = (M + GT_M - 1) / GT_M;
    return (long long)nc * 64 * ((long long)GT_M * (nt - 1) + atc_rows(M, nt - 1));
}

// Split copy of an operator block for the tensor-core GEMM, built on first use
// and shared by every problem list of the context (keyed by the block's
// address, leading dimension and extent); kept in device slabs of 256 MB.
const float *tc_split_operator(hz_ctx *c0, const float2 *A, long long lda, int M, int K) {
    if (!A || M <= 0 || K <= 0) return nullptr;
    hz_ctx *c = c0->parent ? c0->parent : c0;  // lanes share their parent's copies
    const auto key = std::make_tuple((const void *)A, lda, M, K);
    auto it = c->tca.find(key);
    if (it != c->tca.end()) return it->second;
    const long long nf = atc_floats(M, K);
    const size_t bytes = (size_t)nf * 4, align = 512;
    const size_t need = (bytes + align - 1) / align * align;
    if (c->tca_slabs.empty() || c->tca_used + need > c->tca_cap) {
        const size_t cap = std::max<size_t>(need, (size_t)256 << 20);
        c->tca_slabs.push_back(c->dalloc(cap));
        c->tca_cap = cap;
        c->tca_used = 0;
    }
    float *dst = reinterpret_cast<float *>(static_cast<char *>(c->tca_slabs.back()) + c->tca_used);
    c->tca_used += need;
    const long long blocks = std::min<long long>(4096, (nf / 4 + 255) / 256);
    k_build_atc<<<(int)std::max(1LL, blocks), 256, 0, c0->st>>>(A, lda, M, K, dst);
    HZ_CU(cudaGetLastError());
    c0->tca_pending = true;  // the list builder synchronises before the copy is shared
    c->tca[key] = dst;
    return dst;
}

void tc_refresh_operators(hz_ctx *c) {
    for (auto &kv : c->tca) {
        const float2 *A = static_cast<const float2 *>(std::get<0>(kv.first));
        const long long lda = std::get<1>(kv.first);
        const int M = std::get<2>(kv.first), K = std::get<3>(kv.first);
        const long long nf = atc_floats(M, K);
        const long long blocks = std::min<long long>(4096, (nf / 4 + 255) / 256);
        k_build_atc<<<(int)std::max(1LL, blocks), 256, 0, c->st>>>(A, lda, M, K, kv.second);
        HZ_CU(cudaGetLastError());
    }
}

void launch_gemm_tc(const GemmProb<float2> *d_probs, int nprob, int max_tiles, int split, float2 *ws, int *cnt,
                    int *err, cudaStream_t st, int *nl) {
    if (nprob <= 0 || max_tiles <= 0) return;
    if (split < 1 || (split > 1 && (!ws || !cnt))) throw HzError(HZ_EINVAL, "tensor-core GEMM: bad split-K workspace");
    static bool attr = false;
    if (!attr) {
        HZ_CU(cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, GT_SMEM));
        attr = true;
    }
    k_gemm_tc<<<dim3(max_tiles * split, nprob), GT_THREADS, GT_SMEM, st>>>(d_probs, split, ws, cnt, max_tiles, err);
    HZ_CU(cudaGetLastError());
    if (nl) (*nl)++;
}

}  // namespace hz
