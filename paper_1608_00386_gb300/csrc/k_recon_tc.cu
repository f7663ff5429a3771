// Reconstructor product of a batch of realizations on the tensor cores ("The closed loop": slopes
// times the control matrix, here for B independent realizations sharing a bfloat16 R):
//   D[r][i] = sum_j R[i][j] s_r[j],   r < B,
// with R in bfloat16 and the slopes in float32, accumulated in float32.
//
// The tensor cores multiply bfloat16 by bfloat16, so each float32 slope is split exactly into
// three bfloat16 terms, s = hi + mid + lo: hi = bf16(s), mid = bf16(s - hi), lo = bf16(s - hi -
// mid), each difference exact in float32, and the three terms together hold all 24 significand
// bits.  R hi + R mid + R lo is then R s with float32 slopes (every bfloat16 product is exact in
// float32), which is the product the oracle defines for a bfloat16 reconstructor.
//
// Layout.  R is copied once per load into tiles of 128 rows x 64 columns of bfloat16, each tile
// one contiguous 16 KB block, tiles ordered row tile major then k-block: [n_mt][KB][128][64]
// (rows padded to a multiple of 128, columns to a multiple of 64, zeros in the padding).  Each
// step writes the split slopes as [KB][3][npad][64] (realizations past B zero).  A k-block's A
// operand (one tile of R) and B operand (3 npad rows of 64 slopes) are then each one contiguous
// TMA box, K-major with the 128-byte swizzle, and the range of tiles a block streams is one
// contiguous run of memory.  (Boxes of a row-major R touch 128 rows 111 KB apart per k-block;
// that layout streamed at half the rate.)
//
// Kernel.  One persistent block per SM takes a contiguous range of the (row tile, k-block)
// sequence, row tile major, so every block streams the same number of bytes of R; the range
// covers at most a few row tiles (segments).  Warp roles:
//   warp 4, one thread: TMA producer -- cp.async.bulk.tensor loads of both boxes into a ring of
//     stages (R with an L2 evict-first hint: it is read once; the slopes evict-last: every row
//     tile reads them again);
//   warp 5, one thread: MMA issuer -- four tcgen05.mma (M 128, N 3 npad, K 16) per k-block into
//     a TMEM accumulator; a chunk of P.chunk k-blocks (64 columns each) fills one accumulator
//     and up to 8 accumulators (as many as fit the 512 TMEM columns) rotate, so the MMAs run
//     several chunks ahead of the drain; tcgen05.commit frees each stage and, at the end of a
//     chunk, signals its accumulator;
//   warps 0-3: epilogue -- tcgen05.ld of their 32 TMEM lanes (rows), hi + mid + lo per
//     realization, added into float32 registers (round to nearest) chunk after chunk; one
//     partial row sum per (block, segment) in global memory.
// Why chunks: the tensor cores' float32 accumulation is coarser than round-to-nearest.  Over the
// ~3500 MMAs of a whole row tile its error reached 2.3e-5 of the product on random data (39 m
// size); with 32 MMAs per accumulator and a round-to-nearest sum of the chunks it is 5e-7
// (4 MMAs: 3e-7), the float32 accuracy of the CUDA-core path.  Draining every k-block instead
// of every 8 made the product 40 % slower (the drain becomes the serial step).
// A second kernel sums each row tile's partials in block order (deterministic) and applies
// out = alpha D + beta out.  Every mbarrier wait is bounded (about one second of clock); on
// expiry the thread records kErrReconTimeout, stops, and the block drains what it has in flight
// before it frees its TMEM and exits.
#include <cuda.h>

#include <algorithm>
#include <vector>

#include "mcao_internal.h"

namespace mcao {

namespace {

constexpr int kTcM = 128;                 // rows of R per tile = TMEM lanes
constexpr int kTcK = 64;                  // bfloat16 columns per k-block (one 128-byte row)
constexpr int kTcThreads = 192;           // 4 epilogue warps, producer warp, MMA warp
constexpr int kTcMaxRhs = 64;             // realizations per pass
constexpr int kTcMaxStages = 8;
constexpr int kTcChunk = 8;               // k-blocks summed in one TMEM accumulator
constexpr int kTcMaxBufs = 8;             // TMEM accumulators in rotation
constexpr int kTcSmemLimit = 232448;      // 227 KB of dynamic shared memory per block
constexpr long long kTcWaitCycles = 2000000000ll;   // ~1 s at 2 GHz
constexpr uint32_t kABytes = kTcM * kTcK * 2;        // 16 KB per stage of R

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void bar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool bar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// wait for the phase of the given parity to complete, giving up after kTcWaitCycles
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity) {
    if (bar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!bar_try_wait(bar, parity))
        if (clock64() - t0 > kTcWaitCycles) return false;
    return true;
}

__device__ __forceinline__ uint64_t l2_policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// TMA: box at (x = column, y = row) of a 2-D tensor map into shared memory, completing on bar
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar,
                                            uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major operand with the 128-byte swizzle: rows of 128
// bytes, 8-row groups 1024 bytes apart (stride byte offset), start address in 16-byte units,
// descriptor version 1 (bits 46-47), swizzle mode 2 = 128 B (bits 61-63).  The leading byte
// offset is not used by swizzled K-major layouts (set to 1).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of tcgen05.mma kind::f16: float32 accumulator (bits 4-5 = 1), A and B
// bfloat16 (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t bf16_idesc(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// arrive on bar once every tcgen05 operation this thread has issued so far has completed
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 16 consecutive 32-bit TMEM columns of this thread's lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

struct TcParams {
    int KB;             // k-blocks per row tile (ldb / 64)
    long long T;        // row tiles x KB
    int G;              // blocks
    int npad;           // realizations per slope part (multiple of 16)
    int n_rhs;          // realizations of this pass (<= npad)
    int stages;
    int maxseg;         // segments per block, at most
    int chunk;          // k-blocks per TMEM accumulator
    int nbuf;           // TMEM accumulators in rotation
    uint32_t tmem_cols; // allocated TMEM columns (power of two >= nbuf x 3 npad)
    float* partial;     // [G][maxseg][npad][128]
    int* err;
};

struct Seg {
    int m, kb_lo, kb_hi;
};

// k-block range [lo, hi) of block b, split into per-row-tile segments; returns false past the end
__device__ __forceinline__ bool next_seg(long long& p, long long hi, int KB, Seg& s) {
    if (p >= hi) return false;
    const int m = (int)(p / KB);
    const long long end = min(hi, (long long)(m + 1) * KB);
    s.m = m;
    s.kb_lo = (int)(p - (long long)m * KB);
    s.kb_hi = (int)(end - (long long)m * KB);
    p = end;
    return true;
}

__global__ void __launch_bounds__(kTcThreads, 1)
    recon_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcParams P) {
    extern __shared__ unsigned char tc_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tc_raw) + 1023) &
                                                         ~(uintptr_t)1023);
    const uint32_t b_bytes = 3u * (uint32_t)P.npad * kTcK * 2u;
    const uint32_t st_bytes = kABytes + b_bytes;
    const int S = P.stages;
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + (size_t)S * st_bytes);
    uint64_t* empty = full + S;
    uint64_t* tfull = empty + S;          // [nbuf] accumulator ready for the epilogue
    uint64_t* tempty = tfull + P.nbuf;    // [nbuf] accumulator read out, free for the MMA
    uint64_t* drain = tempty + P.nbuf;    // MMA issuer's last commit
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            bar_init(&full[s], 1);
            bar_init(&empty[s], 1);
        }
        for (int b = 0; b < P.nbuf; ++b) {
            bar_init(&tfull[b], 1);
            bar_init(&tempty[b], 4);
        }
        bar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(P.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const long long lo = (long long)blockIdx.x * P.T / P.G;
    const long long hi = (long long)(blockIdx.x + 1) * P.T / P.G;
    const int ncol = 3 * P.npad;   // accumulator columns per segment (hi | mid | lo parts)

    if (warp == 4) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
            const uint64_t pol_a = l2_policy_evict_first(), pol_b = l2_policy_evict_last();
            uint32_t it = 0;
            bool ok = true;
            long long p = lo;
            Seg sg;
            while (ok && next_seg(p, hi, P.KB, sg)) {
                for (int kb = sg.kb_lo; kb < sg.kb_hi; ++kb, ++it) {
                    const int s = (int)(it % (uint32_t)S);
                    const uint32_t round = it / (uint32_t)S;
                    if (!bar_wait(&empty[s], (round & 1u) ^ 1u)) {
                        atomicExch(P.err, kErrReconTimeout);
                        ok = false;
                        break;
                    }
                    unsigned char* a = sm + (size_t)s * st_bytes;
                    bar_expect_tx(&full[s], st_bytes);
                    tma_load_2d(a, &tmA, 0, (int)(((long long)sg.m * P.KB + kb) * kTcM), &full[s], pol_a);
                    tma_load_2d(a + kABytes, &tmB, 0, kb * 3 * P.npad, &full[s], pol_b);
                }
            }
            // every copy issued has landed before the block can exit (bounded)
            const uint32_t first = it > (uint32_t)S ? it - (uint32_t)S : 0u;
            for (uint32_t j = first; j < it; ++j) bar_wait(&full[j % (uint32_t)S], (j / (uint32_t)S) & 1u);
        }
    } else if (warp == 5) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            const uint32_t idesc = bf16_idesc(kTcM, ncol);
            uint32_t it = 0, chunk = 0;
            bool ok = true;
            long long p = lo;
            Seg sg;
            while (ok && next_seg(p, hi, P.KB, sg)) {
                for (int c0 = sg.kb_lo; ok && c0 < sg.kb_hi; c0 += P.chunk, ++chunk) {
                    const int c1 = min(c0 + P.chunk, sg.kb_hi);
                    const uint32_t buf = chunk % (uint32_t)P.nbuf, use = chunk / (uint32_t)P.nbuf;
                    if (!bar_wait(&tempty[buf], (use & 1u) ^ 1u)) {
                        atomicExch(P.err, kErrReconTimeout);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem + buf * (uint32_t)ncol;
                    for (int kb = c0; kb < c1; ++kb, ++it) {
                        const int s = (int)(it % (uint32_t)S);
                        if (!bar_wait(&full[s], (it / (uint32_t)S) & 1u)) {
                            atomicExch(P.err, kErrReconTimeout);
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t a0 = smem_u32(sm + (size_t)s * st_bytes);
                        const uint32_t b0 = a0 + kABytes;
#pragma unroll
                        for (int k = 0; k < kTcK / 16; ++k)
                            tc_mma(d, sw128_desc(a0 + 32u * k), sw128_desc(b0 + 32u * k), idesc,
                                   (kb > c0 || k > 0) ? 1u : 0u);
                        tc_commit(&empty[s]);   // the stage is free once these MMAs have read it
                    }
                    if (!ok) break;
                    tc_commit(&tfull[buf]);
                }
            }
            tc_commit(drain);   // nothing of this thread's is in flight past this wait
            bar_wait(drain, 0u);
        }
    } else {
        // ---------------- epilogue: warp q reads TMEM lanes 32q..32q+31 ----------------
        const int q = warp;
        const int ncg = P.npad / 16;
        uint32_t seg = 0, chunk = 0;
        bool ok = true;
        long long p = lo;
        Seg sg;
        while (ok && next_seg(p, hi, P.KB, sg)) {
            float acc[kTcMaxRhs];
#pragma unroll
            for (int b = 0; b < kTcMaxRhs; ++b) acc[b] = 0.0f;
            for (int c0 = sg.kb_lo; c0 < sg.kb_hi; c0 += P.chunk, ++chunk) {
                const uint32_t buf = chunk % (uint32_t)P.nbuf, use = chunk / (uint32_t)P.nbuf;
                // every lane waits; the warp goes on only if all saw the accumulator (the TMEM
                // loads below must be executed by the whole warp)
                if (!__all_sync(0xffffffffu, bar_wait(&tfull[buf], use & 1u))) {
                    if (lane == 0) atomicExch(P.err, kErrReconTimeout);
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t t0 = tmem + ((uint32_t)(32 * q) << 16) + buf * (uint32_t)ncol;
#pragma unroll
                for (int cg = 0; cg < kTcMaxRhs / 16; ++cg) {
                    if (cg < ncg) {
                        uint32_t vh[16], vm[16], vl[16];
                        tmem_ld16(t0 + 16 * cg, vh);
                        tmem_ld16(t0 + P.npad + 16 * cg, vm);
                        tmem_ld16(t0 + 2 * P.npad + 16 * cg, vl);
                        tmem_wait_ld();
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            acc[16 * cg + i] +=
                                (__uint_as_float(vh[i]) + __uint_as_float(vm[i])) + __uint_as_float(vl[i]);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) bar_arrive(&tempty[buf]);
            }
            if (!ok) break;
            float* out = P.partial + ((size_t)(blockIdx.x * P.maxseg + seg) * P.npad) * kTcM + 32 * q + lane;
#pragma unroll
            for (int b = 0; b < kTcMaxRhs; ++b)
                if (b < P.n_rhs) out[(size_t)b * kTcM] = acc[b];
            ++seg;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(P.tmem_cols)
                     : "memory");
}

// float32 pair -> bfloat16 pair (round to nearest even), x0 in the low half
__device__ __forceinline__ uint32_t bf16x2_rn(float x0, float x1) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(x1), "f"(x0));
    return d;
}
__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

// S[kb][p][b][c] (bfloat16 pairs): the three exact bfloat16 terms p of realization r0 + b's padded
// slope j = 64 kb + c (zero for b >= nb or j >= ld)
__global__ void tc_split_kernel(const float* __restrict__ slopes_pad, int pad_stride, int r0, int nb, int ld,
                                int ldb, int npad, uint32_t* __restrict__ S) {
    const int half = ldb / 2;
    const long long total = (long long)npad * half;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(i / half), jp = (int)(i - (long long)b * half);
        const int j = 2 * jp;
        float x0 = 0.0f, x1 = 0.0f;
        if (b < nb) {
            const float* s = slopes_pad + (long long)(r0 + b) * pad_stride;
            if (j < ld) x0 = s[j];
            if (j + 1 < ld) x1 = s[j + 1];
        }
        const uint32_t h = bf16x2_rn(x0, x1);
        const float r0a = x0 - bf16_lo(h), r0b = x1 - bf16_hi(h);   // exact
        const uint32_t m = bf16x2_rn(r0a, r0b);
        const float r1a = r0a - bf16_lo(m), r1b = r0b - bf16_hi(m);   // exact
        const uint32_t l = bf16x2_rn(r1a, r1b);                        // exact: r1 has <= 8 bits
        const int kb = j / kTcK, c2 = (j - kb * kTcK) / 2;
        const long long base = ((long long)kb * 3 * npad + b) * (kTcK / 2) + c2;   // part 0
        const long long part = (long long)npad * (kTcK / 2);
        S[base] = h;
        S[base + part] = m;
        S[base + 2 * part] = l;
    }
}

// out[r0 + b][row] = alpha sum over the blocks covering row tile row/128 (in block order) of their
// partials + beta out (beta = 0: out not read)
__global__ void tc_reduce_kernel(const float* __restrict__ partial, const int2* __restrict__ cover, long long T, int G,
                                 int KB, int maxseg, int npad, int nb, int r0, int n_cmd, float alpha, float beta,
                                 const float* __restrict__ scale, float* __restrict__ out) {
    const long long total = (long long)nb * n_cmd;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(i / n_cmd), row = (int)(i - (long long)b * n_cmd);
        const int m = row / kTcM, r = row - m * kTcM;
        const int2 cv = cover[m];
        float s = 0.0f;
        for (int blk = cv.x; blk <= cv.y; ++blk) {
            const long long blo = (long long)blk * T / G;
            const int seg = m - (int)(blo / KB);
            s += partial[((size_t)(blk * maxseg + seg) * npad + b) * kTcM + r];
        }
        if (scale) s *= scale[row];   // FP8 E4M3: the row's scale times its code-value sum
        float* o = out + (long long)(r0 + b) * n_cmd + row;
        *o = beta == 0.0f ? alpha * s : fmaf(alpha, s, beta * *o);
    }
}

// row-major float32 [rows_in][ld] -> bfloat16 tiles [n_mt][KB][128][64] (rows x ldb in all),
// zero padding
__global__ void tc_pack_kernel(const float* __restrict__ src, int rows_in, int ld, int rows, int ldb,
                               uint32_t* __restrict__ dst) {
    const int half = ldb / 2;
    const int KB = ldb / kTcK;
    const long long total = (long long)rows * half;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        // i enumerates the destination: tile (m, kb), row r in the tile, column pair c2
        const long long tile = i / (kTcM * (kTcK / 2));
        const int in_tile = (int)(i - tile * (kTcM * (kTcK / 2)));
        const int r = in_tile / (kTcK / 2), c2 = in_tile - r * (kTcK / 2);
        const int m = (int)(tile / KB), kb = (int)(tile - (long long)m * KB);
        const int row = m * kTcM + r, j = kb * kTcK + 2 * c2;
        float x0 = 0.0f, x1 = 0.0f;
        if (row < rows_in) {
            if (j < ld) x0 = src[(long long)row * ld + j];
            if (j + 1 < ld) x1 = src[(long long)row * ld + j + 1];
        }
        dst[i] = bf16x2_rn(x0, x1);
    }
}

// FP8 E4M3 R: code = e4m3(fl(R / scale_row)) (round to nearest even, saturating), the stored
// format's own rule; its value is exact in bfloat16, so the tiles hold the code values and the
// reduction multiplies each row sum by the row's scale
__device__ __forceinline__ float e4m3_value(float x, float scale) {
    const float q = __fdiv_rn(x, scale);
    uint16_t code;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(code) : "f"(0.0f), "f"(q));
    uint32_t h2;
    asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(h2) : "h"(code));
    float v;
    asm("{\n\t.reg .f16 a, b;\n\tmov.b32 {a, b}, %1;\n\tcvt.f32.f16 %0, a;\n\t}" : "=f"(v) : "r"(h2));
    return v;
}

__global__ void tc_pack_e4m3_kernel(const float* __restrict__ src, int rows_in, int ld, int rows, int ldb,
                                    const float* __restrict__ scale, uint32_t* __restrict__ dst) {
    const int half = ldb / 2;
    const int KB = ldb / kTcK;
    const long long total = (long long)rows * half;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long tile = i / (kTcM * (kTcK / 2));
        const int in_tile = (int)(i - tile * (kTcM * (kTcK / 2)));
        const int r = in_tile / (kTcK / 2), c2 = in_tile - r * (kTcK / 2);
        const int m = (int)(tile / KB), kb = (int)(tile - (long long)m * KB);
        const int row = m * kTcM + r, j = kb * kTcK + 2 * c2;
        float x0 = 0.0f, x1 = 0.0f;
        if (row < rows_in) {
            const float sc = scale[row];
            if (j < ld) x0 = e4m3_value(src[(long long)row * ld + j], sc);
            if (j + 1 < ld) x1 = e4m3_value(src[(long long)row * ld + j + 1], sc);
        }
        dst[i] = bf16x2_rn(x0, x1);   // exact: an E4M3 value has at most 4 significant bits
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// 2-D bfloat16 tensor map of a row-major [rows][cols] array, box [box_rows][64], 128-byte swizzle
bool make_map(CUtensorMap* map, const void* base, long long rows, long long cols, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {(cuuint32_t)kTcK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

struct TcProduct {
    CUtensorMap tmA, tmB;
    uint16_t* R = nullptr;       // [n_mt][KB][128][64]
    uint16_t* S = nullptr;       // [KB][3][npad][64]
    float* partial = nullptr;    // [G][maxseg][npad][128]
    float* scale = nullptr;      // [rows]: FP8 E4M3 row scales (null for bfloat16)
    int2* cover = nullptr;       // [n_mt] first and last block of each row tile
    int n_cmd = 0, rows = 0, ld = 0, ldb = 0, n_mt = 0, KB = 0, G = 0, npad = 0, stages = 0, maxseg = 0, nbuf = 0;
    uint32_t tmem_cols = 0;
    long long T = 0;
    size_t smem = 0;
};

void tc_destroy(TcProduct* P) {
    if (!P) return;
    cudaFree(P->R);
    cudaFree(P->S);
    cudaFree(P->partial);
    cudaFree(P->cover);
    cudaFree(P->scale);
    delete P;
}

cudaError_t tc_create(const float* R_rm, int rows_in, int ld, int n_cmd, int n_rhs, int sm_count, int fp8,
                      cudaStream_t st, TcProduct** out) {
    *out = nullptr;
    if (n_cmd < 1 || ld < 1 || n_rhs < 1 || rows_in < n_cmd) return cudaErrorInvalidValue;
    TcProduct* P = new TcProduct();
    P->n_cmd = n_cmd;
    P->ld = ld;
    P->rows = (n_cmd + kTcM - 1) / kTcM * kTcM;
    P->ldb = (ld + kTcK - 1) / kTcK * kTcK;
    P->n_mt = P->rows / kTcM;
    P->KB = P->ldb / kTcK;
    P->T = (long long)P->n_mt * P->KB;
    P->G = (int)std::min<long long>(std::max(sm_count, 1), P->T);
    P->npad = (std::min(n_rhs, kTcMaxRhs) + 15) / 16 * 16;
    const size_t st_bytes = kABytes + 3u * (size_t)P->npad * kTcK * 2u;
    const size_t tail = 1024 + (2 * kTcMaxStages + 2 * kTcMaxBufs + 1) * sizeof(uint64_t) + 16;
    P->stages = (int)std::min<size_t>(kTcMaxStages, (kTcSmemLimit - tail) / st_bytes);
    P->smem = (size_t)P->stages * st_bytes + tail;
    P->nbuf = std::min(kTcMaxBufs, 512 / (3 * P->npad));
    uint32_t cols = 32;
    while (cols < (uint32_t)P->nbuf * 3u * (uint32_t)P->npad) cols *= 2;
    P->tmem_cols = cols;
    // segments per block and the blocks covering each row tile
    std::vector<int2> cover(P->n_mt, make_int2(P->G, -1));
    P->maxseg = 1;
    for (int b = 0; b < P->G; ++b) {
        const long long lo = (long long)b * P->T / P->G, hi = (long long)(b + 1) * P->T / P->G;
        if (hi <= lo) continue;
        const int m0 = (int)(lo / P->KB), m1 = (int)((hi - 1) / P->KB);
        P->maxseg = std::max(P->maxseg, m1 - m0 + 1);
        for (int m = m0; m <= m1; ++m) {
            cover[m].x = std::min(cover[m].x, b);
            cover[m].y = std::max(cover[m].y, b);
        }
    }
    cudaError_t e = cudaMalloc(&P->R, sizeof(uint16_t) * (size_t)P->rows * P->ldb);
    if (e == cudaSuccess) e = cudaMalloc(&P->S, sizeof(uint16_t) * 3 * (size_t)P->npad * P->ldb);
    if (e == cudaSuccess)
        e = cudaMalloc(&P->partial, sizeof(float) * (size_t)P->G * P->maxseg * P->npad * kTcM);
    if (e == cudaSuccess) e = cudaMalloc(&P->cover, sizeof(int2) * P->n_mt);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(P->cover, cover.data(), sizeof(int2) * P->n_mt, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && fp8) {
        e = cudaMalloc(&P->scale, sizeof(float) * (size_t)std::max(P->rows, rows_in));
        if (e == cudaSuccess) e = launch_recon_scales(R_rm, rows_in, ld, ld, P->scale, st);
        if (e == cudaSuccess) {
            tc_pack_e4m3_kernel<<<2048, 256, 0, st>>>(R_rm, rows_in, ld, P->rows, P->ldb, P->scale,
                                                      reinterpret_cast<uint32_t*>(P->R));
            e = cudaGetLastError();
        }
    } else if (e == cudaSuccess) {
        tc_pack_kernel<<<2048, 256, 0, st>>>(R_rm, rows_in, ld, P->rows, P->ldb, reinterpret_cast<uint32_t*>(P->R));
        e = cudaGetLastError();
    }
    // both maps see their array as 64-column rows: a box is box_rows consecutive rows, i.e. one
    // contiguous block
    if (e == cudaSuccess && (!make_map(&P->tmA, P->R, (long long)P->rows * P->KB, kTcK, kTcM) ||
                             !make_map(&P->tmB, P->S, (long long)P->KB * 3 * P->npad, kTcK, 3 * P->npad)))
        e = cudaErrorNotSupported;
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(recon_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P->smem);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        tc_destroy(P);
        return e;
    }
    *out = P;
    return cudaSuccess;
}

long long tc_bytes(const TcProduct* P) { return P ? (long long)P->rows * P->ldb * 2 : 0; }

cudaError_t tc_launch(TcProduct* P, const float* slopes_pad, int pad_stride, int n_real, float alpha, float beta,
                      float* out, int* err, int chunk, cudaStream_t st, int* launches) {
    int nl = 0;
    for (int r0 = 0; r0 < n_real; r0 += P->npad) {
        const int nb = std::min(P->npad, n_real - r0);
        const long long pairs = (long long)P->npad * (P->ldb / 2);
        const int split_blocks = (int)std::min<long long>(1024, (pairs + 255) / 256);
        tc_split_kernel<<<split_blocks, 256, 0, st>>>(slopes_pad, pad_stride, r0, nb, P->ld, P->ldb, P->npad,
                                                      reinterpret_cast<uint32_t*>(P->S));
        TcParams prm;
        prm.KB = P->KB;
        prm.T = P->T;
        prm.G = P->G;
        prm.npad = P->npad;
        prm.n_rhs = nb;
        prm.stages = P->stages;
        prm.maxseg = P->maxseg;
        prm.chunk = chunk > 0 ? chunk : kTcChunk;
        prm.nbuf = P->nbuf;
        prm.tmem_cols = P->tmem_cols;
        prm.partial = P->partial;
        prm.err = err;
        recon_tc_kernel<<<P->G, kTcThreads, P->smem, st>>>(P->tmA, P->tmB, prm);
        const long long tot = (long long)nb * P->n_cmd;
        tc_reduce_kernel<<<(int)std::min<long long>(4096, (tot + 255) / 256), 256, 0, st>>>(
            P->partial, P->cover, P->T, P->G, P->KB, P->maxseg, P->npad, nb, r0, P->n_cmd, alpha, beta, P->scale, out);
        nl += 3;
    }
    if (launches) *launches = nl;
    return cudaGetLastError();
}

}  // namespace mcao
