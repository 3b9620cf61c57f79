// Tensor-core form of the cell chain (mixed precision, sm_103a tcgen05).
//
// The cell solve of Alg. inner_solver is the block-tridiagonal chain
//   y_0 = W_0 g_0,  y_j = W_j (g_j - cz_{j-1} . y_{j-1}),
//   x_{nz-1} = y_{nz-1},  x_j = y_j - W_j (cz_j . x_{j+1}),
// i.e. one dense complex product D = W_j T per step, T being the nx x NT
// panel of right-hand sides (NT = 32 or 64) the previous step's epilogue
// produced.  Here every product runs on the 5th-generation tensor cores as
// four real products
// (Wr Tr, Wi Ti, Wr Ti, Wi Tr), each with the 3xTF32 split
// X Y ~ Xh Yh + Xh Yl + Xl Yh (Xh = X rounded to TF32, Xl = X - Xh rounded to
// TF32), which keeps the product accurate to about FP32 roundoff:
//   - W_j is split offline (from the FP64 factors) into Wr_h, Wr_l, Wi_h,
//     Wi_l, stored in the no-swizzle K-major canonical layout of the MMA
//     operand, 16 columns per chunk, so a chunk is one contiguous bulk (TMA)
//     copy; chunks stream through a shared-memory ring (4 stages with
//     NT = 32, 3 with NT = 64; mbarriers "full" / "empty");
//   - T is kept in shared memory as Tr_h, Tr_l, Ti_h, Ti_l in the same
//     canonical layout (rows = right-hand sides, K = cell columns);
//   - a producer warp streams the W chunks through the ring ahead of use;
//     one thread issues the tcgen05.mma instructions (M = 128 rows of W,
//     N = NT right-hand sides, K = 8 per instruction) into FP32 accumulators
//     in tensor memory (the small cross terms apart from the main Xh Yh
//     terms; with NT = 32 also the main terms of even and odd K chunks apart)
//     and commits them to mbarriers;
//   - the 128 threads (thread = row of W, = TMEM lane) read the accumulators
//     with tcgen05.ld, form the step's output (stored to global memory) and
//     the next T, split it and write it back through a per-warp transpose.
// One CTA per (cell, NT right-hand sides); cells up to 128 columns wide.
// Every wait is bounded (1 s): a timeout sets the error word and the whole
// CTA leaves the steps together, drains its bulk copies and frees its tensor
// memory before it returns.
#include "hz_tc.cuh"

namespace hz {

namespace {

constexpr int TC_KC = 16;    // K columns per streamed chunk
constexpr int TC_ST = 4;     // ring stages
constexpr int TC_THREADS = 160;  // warps 0-3: MMA issue and epilogue (TMEM lanes 0-127); warp 4: producer
constexpr int TC_STAGE_BYTES = 4 * 16 * (TC_KC / 4) * 128;  // 4 arrays x 16 row groups x SBO

// Build the split W blocks of every cell (see the file header).  Per cell at
// tc_off (floats): per block j: chunks c of KC_c = min(16, Kp - 16c) columns,
// each [Wr_h, Wr_l, Wi_h, Wi_l][8 R8 rows x KC_c] canonical (rows >= nx and
// columns >= nx are zero), Kp = 8 R8, R8 = ceil(nx / 8).
__global__ void k_build_wtc(const CellDesc *__restrict__ cells, const double2 *__restrict__ W, float *wtc) {
    const CellDesc cd = cells[blockIdx.y];
    const int nx = cd.nx, R8 = (nx + 7) / 8, Kp = 8 * R8, rows = 8 * R8;
    const long long per_block = 32LL * R8 * Kp;
    const long long n = (long long)cd.nz * rows * Kp;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e % Kp);
        const int r = (int)((e / Kp) % rows);
        const int j = (int)(e / ((long long)Kp * rows));
        double2 w = make_double2(0.0, 0.0);
        if (r < nx && k < nx) w = W[cd.w_off + ((long long)j * nx + r) * cd.ldw + k];
        const float rh = tf32_rna((float)w.x), ih = tf32_rna((float)w.y);
        const float rl = tf32_rna((float)(w.x - (double)rh)), il = tf32_rna((float)(w.y - (double)ih));
        const int c = k / TC_KC, kc = k % TC_KC, KC = min(TC_KC, Kp - c * TC_KC);
        float *chunk = wtc + cd.tc_off + j * per_block + (long long)c * 4 * rows * TC_KC;
        const long long arr = (long long)rows * KC;  // floats per array in this chunk
        const unsigned off = canon(r, kc, KC) / 4;
        chunk[off] = rh;
        chunk[arr + off] = rl;
        chunk[2 * arr + off] = ih;
        chunk[3 * arr + off] = il;
    }
}

// Write 16 values per thread (thread = K index k = 32 warp + lane, values for
// right-hand sides n0..n0+15) into a canonical T array [32 rows = n][Kp],
// through a per-warp transpose so that every store is 16 bytes.
__device__ __forceinline__ void put_T(float *Tq, int kext, int n0, const float (&v)[16], float *scr, int warp,
                                      int lane) {
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 16; i++) scr[lane * 33 + i] = v[i];
    __syncwarp();
    const int nl = lane & 15;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const int kg = (lane >> 4) + 2 * q;  // 4-column group within the warp's 32 K values
        float4 w;
        w.x = scr[(4 * kg + 0) * 33 + nl];
        w.y = scr[(4 * kg + 1) * 33 + nl];
        w.z = scr[(4 * kg + 2) * 33 + nl];
        w.w = scr[(4 * kg + 3) * 33 + nl];
        const int k = 32 * warp + 4 * kg;
        if (k < kext) *reinterpret_cast<float4 *>(reinterpret_cast<char *>(Tq) + canon(n0 + nl, k, kext)) = w;
    }
}

// NT right-hand sides per CTA (MMA N): 32 (12 accumulators, the main terms of even
// and odd K chunks apart, 4 ring stages) or 64 (8 accumulators, 3 ring stages;
// the W stream then serves twice the right-hand sides)
template <int NT>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_cell_chain_tc(const CellDesc *__restrict__ cells, const float *__restrict__ wtc, const float2 *__restrict__ cz,
                    float2 *vol, int B, int *err) {
    constexpr int ST = NT == 64 ? 3 : TC_ST;         // ring stages
    constexpr int NACC = NT == 64 ? 8 : 12;          // accumulators of NT columns (NACC * NT <= 512)
    extern __shared__ __align__(1024) unsigned char smraw[];
    __shared__ __align__(8) unsigned long long full[ST], empty[ST], done;
    __shared__ unsigned tmem_slot;
    __shared__ volatile int s_dead;
    __shared__ int s_loaded;  // chunks the producer issued
    const CellDesc cd = cells[blockIdx.y];
    const int nx = cd.nx, nz = cd.nz;
    const int n0 = blockIdx.x * NT;
    if (n0 >= B) return;  // uniform
    const int R8 = (nx + 7) / 8, Kp = 8 * R8, rows = 8 * R8;
    const int nchk = (Kp + TC_KC - 1) / TC_KC;
    const int nsteps = 2 * nz - 1, total = nsteps * nchk;
    const long long per_block = 32LL * R8 * Kp;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char *ring = smraw;
    float *T = reinterpret_cast<float *>(smraw + ST * TC_STAGE_BYTES);  // Tr_h, Tr_l, Ti_h, Ti_l
    const int tarr = NT * Kp;                                          // floats per T array
    float *scr = T + 4 * tarr + (warp & 3) * 32 * 33;
    const float *wc = wtc + cd.tc_off;
    const float2 *czc = cz + cd.cz_off;
    float2 *v = vol + cd.vol_off * (long long)B;
    const long long rs = (long long)nx * B;
    auto jb_of = [&](int s) { return s < nz ? s : 2 * nz - 2 - s; };
    auto chunk_kc = [&](int c) { return min(TC_KC, Kp - c * TC_KC); };
    auto load = [&](int q) {  // producer lane
        const int s = q / nchk, c = q % nchk, st = q % ST;
        const unsigned bytes = (unsigned)(4 * rows * chunk_kc(c) * 4);
        const float *src = wc + jb_of(s) * per_block + (long long)c * 4 * rows * TC_KC;
        mb_expect(su32(&full[st]), bytes);
        bulk_g2s(su32(ring + st * TC_STAGE_BYTES), src, bytes, su32(&full[st]));
    };
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_slot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < ST; i++) {
            mb_init(su32(&full[i]), 1);
            mb_init(su32(&empty[i]), 1);
        }
        mb_init(su32(&done), 1);
        s_dead = 0;
        s_loaded = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // this thread's row of the panel (K index of T, row of W and of D); warps 0-3
    const int m = tid;
    const bool mrow = warp < 4 && m < nx;
    if (warp < 4) {  // t_0 = g_0
        float tr[NT / 16][16], ti[NT / 16][16];
#pragma unroll
        for (int h = 0; h < NT / 16; h++)
#pragma unroll
            for (int i = 0; i < 16; i++) {
                const int n = 16 * h + i;
                float2 g = make_float2(0.f, 0.f);
                if (mrow && n0 + n < B) g = v[(long long)m * B + n0 + n];
                tr[h][i] = g.x;
                ti[h][i] = g.y;
            }
#pragma unroll
        for (int h = 0; h < NT / 16; h++) {
            float a[16], b[16];
#pragma unroll
            for (int i = 0; i < 16; i++) {
                a[i] = tf32_rna(tr[h][i]);
                b[i] = tf32_rna(tr[h][i] - a[i]);
            }
            put_T(T, Kp, 16 * h, a, scr, warp, lane);
            put_T(T + tarr, Kp, 16 * h, b, scr, warp, lane);
#pragma unroll
            for (int i = 0; i < 16; i++) {
                a[i] = tf32_rna(ti[h][i]);
                b[i] = tf32_rna(ti[h][i] - a[i]);
            }
            put_T(T + 2 * tarr, Kp, 16 * h, a, scr, warp, lane);
            put_T(T + 3 * tarr, Kp, 16 * h, b, scr, warp, lane);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = tmem_slot;
    bool dead = false;
    int q_waited = 0;  // thread 0: chunks whose data it has consumed
    if (warp == 4) {
        // producer: streams the W chunks of every step through the ring, ST ahead
        if (lane == 0) {
            for (int q = 0; q < total; q++) {
                const int st = q % ST;
                if (q >= ST && !mb_wait(su32(&empty[st]), (unsigned)(((q / ST) - 1) & 1), dead, err)) {
                    s_dead = 1;
                    break;
                }
                if (s_dead) break;
                load(q);
                s_loaded = q + 1;
            }
        }
        __syncwarp();  // the warp reaches the block barrier below converged
    } else {
        // D accumulators (NT columns each): main terms Xh Yh of P1 = Wr Tr, P2 = Wi Ti,
        // P3 = Wr Ti, P4 = Wi Tr at columns 0..4NT-1 (NT = 32: even K chunks there, odd
        // chunks at 128..255), cross terms Xh Yl + Xl Yh at 256..256+4NT-1.  Short chains
        // of additions into each accumulator keep the tensor core's truncating
        // accumulation small.
        const unsigned idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(NT >> 3) << 17) | (8u << 24);
        const unsigned sboT = (unsigned)(Kp / 4) * 128;
        const unsigned tbase = su32(T);
        for (int s = 0; s < nsteps; s++) {
            const bool fwd = s < nz;
            const int jb = jb_of(s);
            if (tid == 0 && !dead) {
                for (int c = 0; c < nchk && !dead; c++) {
                    const int q = s * nchk + c, st = q % ST;
                    if (!mb_wait(su32(&full[st]), (unsigned)((q / ST) & 1), dead, err)) break;
                    q_waited = q + 1;
                    tc_fence_after();
                    const int KC = chunk_kc(c);
                    const unsigned sbo = (unsigned)(KC / 4) * 128;
                    const unsigned abase = su32(ring + st * TC_STAGE_BYTES);
                    const unsigned arr = (unsigned)(rows * KC * 4);  // bytes per W array in this chunk
                    const unsigned long long dW = sdesc(abase, 128, sbo), dT = sdesc(tbase, 128, sboT);
                    const unsigned mainc = (NT == 32 && (c & 1)) ? 128u : 0u;
                    for (int t = 0; t < KC / 8; t++) {
                        const int k0 = c * TC_KC + 8 * t;
                        // first product into a main accumulator (NT = 32: even and odd chunks apart)
                        const unsigned fm = ((NT == 32 ? c < 2 : c == 0) && t == 0) ? 0u : 1u;
                        const unsigned fx = (c == 0 && t == 0) ? 0u : 1u;  // first product into a cross accumulator
                        const unsigned long long aoff = (unsigned long long)((t * 256u) >> 4);
                        const unsigned long long Wrh = dW + aoff, Wrl = dW + aoff + ((1u * arr) >> 4);
                        const unsigned long long Wih = dW + aoff + ((2u * arr) >> 4), Wil = dW + aoff + ((3u * arr) >> 4);
                        const unsigned long long toff = (unsigned long long)((((unsigned)k0 / 4) * 128u) >> 4);
                        const unsigned long long tq = (unsigned long long)(((unsigned)tarr * 4u) >> 4);
                        const unsigned long long Trh = dT + toff, Trl = dT + toff + tq, Tih = dT + toff + 2 * tq,
                                                 Til = dT + toff + 3 * tq;
                        umma_tf32(tmem + mainc + 0 * NT, Wrh, Trh, idesc, fm);  // P1 main
                        umma_tf32(tmem + mainc + 1 * NT, Wih, Tih, idesc, fm);  // P2 main
                        umma_tf32(tmem + mainc + 2 * NT, Wrh, Tih, idesc, fm);  // P3 main
                        umma_tf32(tmem + mainc + 3 * NT, Wih, Trh, idesc, fm);  // P4 main
                        umma_tf32(tmem + 256 + 0 * NT, Wrh, Trl, idesc, fx);    // P1 cross
                        umma_tf32(tmem + 256 + 0 * NT, Wrl, Trh, idesc, 1u);
                        umma_tf32(tmem + 256 + 1 * NT, Wih, Til, idesc, fx);    // P2 cross
                        umma_tf32(tmem + 256 + 1 * NT, Wil, Tih, idesc, 1u);
                        umma_tf32(tmem + 256 + 2 * NT, Wrh, Til, idesc, fx);    // P3 cross
                        umma_tf32(tmem + 256 + 2 * NT, Wrl, Tih, idesc, 1u);
                        umma_tf32(tmem + 256 + 3 * NT, Wih, Trl, idesc, fx);    // P4 cross
                        umma_tf32(tmem + 256 + 3 * NT, Wil, Trh, idesc, 1u);
                    }
                    umma_commit(su32(&empty[st]));  // the producer may refill this stage once these are done
                }
                if (!dead) umma_commit(su32(&done));
            }
            // global vector of this step's epilogue (forward: g of step s+1; backward: y of
            // step s), row m, loaded one 8-column quarter ahead of its use
            const int sg = fwd ? (s + 1 < nz ? s + 1 : -1) : s;
            const float2 *gsrc = (sg >= 0 && mrow) ? v + jb_of(sg) * rs + (long long)m * B + n0 : nullptr;
            auto gload = [&](int q8, float2 (&gq)[8]) {
#pragma unroll
                for (int i = 0; i < 8; i++) {
                    const int n = 8 * q8 + i;
                    gq[i] = (gsrc && n0 + n < B) ? gsrc[n] : make_float2(0.f, 0.f);
                }
            };
            float2 gcur[8], gnext[8];
            gload(0, gcur);
            const float2 c_out = (mrow && fwd && s + 1 < nz) ? czc[(long long)jb * nx + m] : make_float2(0.f, 0.f);
            const float2 c_next = (mrow && jb > 0) ? czc[(long long)(jb - 1) * nx + m] : make_float2(0.f, 0.f);
            if (!dead) mb_wait(su32(&done), (unsigned)(s & 1), dead, err);
            __syncwarp();
            const bool wdead = __any_sync(0xffffffffu, dead);
            if (!wdead) {
                tc_fence_after();
                float2 *g = v + jb * rs + (long long)m * B + n0;
#pragma unroll
                for (int h = 0; h < NT / 16; h++) {
                    float nr[16], ni[16];
#pragma unroll
                    for (int qq = 0; qq < 2; qq++) {
                        const int q8 = 2 * h + qq;
                        if (q8 + 1 < NT / 8) gload(q8 + 1, gnext);
                        float p[NACC][8];
                        const unsigned ta = tmem + ((unsigned)(32 * warp) << 16) + 8 * q8;
#pragma unroll
                        for (int a = 0; a < NACC; a++) tmem_ld8(ta + NT * a, p[a]);
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                        if (NT == 32 && nchk < 2) {  // no odd chunks: those accumulators were never written
#pragma unroll
                            for (int a = 4; a < 8; a++)
#pragma unroll
                                for (int i = 0; i < 8; i++) p[a][i] = 0.f;
                        }
#pragma unroll
                        for (int i = 0; i < 8; i++) {
                            const int n = 8 * q8 + i;
                            float s1, s2, s3, s4;  // P1..P4: main (+ odd-chunk main) + cross
                            if (NT == 32) {
                                s1 = (p[0][i] + p[4][i]) + p[8][i];
                                s2 = (p[1][i] + p[5][i]) + p[9][i];
                                s3 = (p[2][i] + p[6][i]) + p[10][i];
                                s4 = (p[3][i] + p[7][i]) + p[11][i];
                            } else {
                                s1 = p[0][i] + p[4][i];
                                s2 = p[1][i] + p[5][i];
                                s3 = p[2][i] + p[6][i];
                                s4 = p[3][i] + p[7][i];
                            }
                            float2 out = make_float2(s1 - s2, s3 + s4);
                            float2 tn;
                            if (fwd) {
                                if (s + 1 < nz)
                                    tn = gcur[i] - c_out * out;  // g_{j+1} - c_j y_j
                                else
                                    tn = c_next * out;  // first backward step: c_{nz-2} x_{nz-1}
                            } else {
                                out = gcur[i] - out;  // x_j = y_j - W_j t
                                tn = c_next * out;
                            }
                            const bool live = mrow && n0 + n < B;
                            if (!live) {
                                out = make_float2(0.f, 0.f);
                                tn = make_float2(0.f, 0.f);
                            } else {
                                g[n] = out;
                            }
                            nr[8 * qq + i] = tn.x;
                            ni[8 * qq + i] = tn.y;
                        }
#pragma unroll
                        for (int i = 0; i < 8; i++) gcur[i] = gnext[i];
                    }
                    float a[16], b[16];
#pragma unroll
                    for (int i = 0; i < 16; i++) {
                        a[i] = tf32_rna(nr[i]);
                        b[i] = tf32_rna(nr[i] - a[i]);
                    }
                    put_T(T, Kp, 16 * h, a, scr, warp, lane);
                    put_T(T + tarr, Kp, 16 * h, b, scr, warp, lane);
#pragma unroll
                    for (int i = 0; i < 16; i++) {
                        a[i] = tf32_rna(ni[i]);
                        b[i] = tf32_rna(ni[i] - a[i]);
                    }
                    put_T(T + 2 * tarr, Kp, 16 * h, a, scr, warp, lane);
                    put_T(T + 3 * tarr, Kp, 16 * h, b, scr, warp, lane);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // T written by threads -> read by the MMAs
            tc_fence_before();
            if (dead) s_dead = 1;
            asm volatile("bar.sync 1, 128;" ::: "memory");  // warps 0-3 only: the producer runs on
            if (s_dead) {
                dead = true;
                break;
            }
            tc_fence_after();
        }
        if (dead) s_dead = 1;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // after a timeout: let the bulk copies issued for this CTA land before it leaves
    if (tid == 0 && s_dead) {
        for (int q = q_waited; q < s_loaded; q++)
            mb_wait(su32(&full[q % ST]), (unsigned)((q / ST) & 1), dead, err);
    }
    __syncthreads();
    if (s_dead) __nanosleep(20000);  // products still in flight finish before the tensor memory is freed
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

}  // namespace

static size_t tc_smem(int nt, int max_nx) {
    const int Kp = 8 * ((max_nx + 7) / 8);
    const int st = nt == 64 ? 3 : TC_ST;
    return (size_t)st * TC_STAGE_BYTES + (size_t)4 * nt * Kp * 4 + (size_t)4 * 32 * 33 * 4;
}
size_t cell_chain_tc_smem(int max_nx) { return tc_smem(32, max_nx); }

long long cell_tc_floats(int nx, int nz) {
    const int R8 = (nx + 7) / 8;
    return (long long)nz * 32 * R8 * (8 * R8);
}

void build_wtc(const CellDesc *d_cells, int ncell, const double2 *W, float *wtc, cudaStream_t st, int *nl) {
    if (ncell <= 0) return;
    k_build_wtc<<<dim3(256, ncell), 256, 0, st>>>(d_cells, W, wtc);
    HZ_CU(cudaGetLastError());
    if (nl) (*nl)++;
}

void launch_cell_chain_tc(const CellDesc *d_cells, int ncell, const float *wtc, const float2 *cz, float2 *vol, int B,
                          int max_nx, int *err, cudaStream_t st, int *nl) {
    if (ncell <= 0 || B <= 0) return;
    if (max_nx > 128) throw HzError(HZ_EINVAL, "tensor-core cell solve: cells wider than 128 columns");
    // 64 right-hand sides per CTA when the batch has more than 32 and the panel fits
    const bool wide = B > 32 && tc_smem(64, max_nx) <= 220 * 1024;
    const size_t sm = tc_smem(wide ? 64 : 32, max_nx);
    if (wide) {
        HZ_CU(cudaFuncSetAttribute(k_cell_chain_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_cell_chain_tc<64><<<dim3((B + 63) / 64, ncell), TC_THREADS, sm, st>>>(d_cells, wtc, cz, vol, B, err);
    } else {
        HZ_CU(cudaFuncSetAttribute(k_cell_chain_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_cell_chain_tc<32><<<dim3((B + 31) / 32, ncell), TC_THREADS, sm, st>>>(d_cells, wtc, cz, vol, B, err);
    }
    HZ_CU(cudaGetLastError());
    if (nl) (*nl)++;
}

// Timeout check: one warp; lane 0 initialises an mbarrier that expects one
// arrival nobody makes and waits for it through the library's bounded wait,
// which runs out after the context's limit and sets the error word.  Nothing
// asynchronous is in flight, so the block simply ends.
__global__ void k_wait_check(int *err) {
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x == 0) {
        mb_init(su32(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        bool dead = false;
        mb_wait(su32(&bar), 0u, dead, err);
    }
}

void launch_wait_check(int *err, cudaStream_t st, int *nl) {
    k_wait_check<<<1, 32, 0, st>>>(err);
    HZ_CU(cudaGetLastError());
    if (nl) (*nl)++;
}

}  // namespace hz
