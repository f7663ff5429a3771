// Reconstructor product and integrator ("The closed loop" of arXiv:1608.00386: slopes times the
// control matrix give differential coefficients added to the mirror commands; pure integrator):
//   Delta c = R s,   c <- c + g Delta c.
// R is float32 [n_cmd][n_slopes], far larger than L2, and is read exactly once per step, so the
// product is bound by HBM bandwidth.  The product is issued per slice of columns (one slice per
// wavefront sensor, so a slice can start as soon as its sensor's slopes exist) and split-K
// inside a slice: a work item is 4 rows times one column chunk; row sums go to a partial buffer
// [n_chunks][n_cmd], and a second kernel adds the partials in a fixed order (deterministic) and
// applies the gain.  The slopes are read (L1-cached) from a copy the sensing kernels write in
// R's padded column layout, so every 16-byte load of s is aligned.
//
// Formats.  R is stored as float32, bfloat16 or FP8 E4M3 with one float scale per row (the
// reduced-precision variants); elements move in 16-byte vectors and are widened to float32 in
// registers, the slopes stay float32, accumulation is float32 and an E4M3 row sum is multiplied
// by its row's scale before it is written.
//
// Streaming.  At most one block per SM (5 warps).  Each warp owns a two-stage ring in
// shared memory and keeps it filled with TMA bulk copies (cp.async.bulk, completion counted on a
// per-stage mbarrier, L2 evict-first policy).  R is held stage-tiled (see ReconLaunch), so each
// stage -- four row segments of up to 2 KB -- is one contiguous copy of up to 8 KB (bulk copies
// that small lose bandwidth), and up to 80 KB per SM are in flight.  The block needs
// few registers and warps, which leaves each SM room for three wavefront-sensor blocks that run
// concurrently, hiding their ALU work under the HBM stream.  Inside the step, five warps with
// two stages each stream faster than three with four (same or less shared memory): the block's
// warps compete for issue slots with the co-resident sensing warps, and more of them get more
// turns; rings above 96 KB keep the science kernels off the SM and slow the step.  Every mbarrier wait is bounded
// (about one second of clock); on expiry the warp records kErrReconTimeout, waits (bounded)
// for its copies in flight and exits.
#include "mcao_internal.h"

namespace mcao {

namespace {

constexpr int kKC = kReconChunk;

// packed FP32 multiply-add (two lanes of a 64-bit register pair per instruction):
// (c.x, c.y) + (a.x b.x, a.y b.y), each rounded once
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
    unsigned long long d;
    asm("{\n\t.reg .b64 ra, rb, rc;\n\tmov.b64 ra, {%1, %2};\n\tmov.b64 rb, {%3, %4};\n\t"
        "mov.b64 rc, {%5, %6};\n\tfma.rn.f32x2 %0, ra, rb, rc;\n\t}"
        : "=l"(d)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(d));
    return r;
}

// even and odd products of a float4 pair accumulated in the two halves of acc
__device__ __forceinline__ float2 dot4x2(float4 a, float4 b, float2 acc) {
    acc = ffma2(make_float2(a.x, a.y), make_float2(b.x, b.y), acc);
    return ffma2(make_float2(a.z, a.w), make_float2(b.z, b.w), acc);
}

// ------------------------------------------------------------------------------------------
// TMA bulk-copy streaming
// ------------------------------------------------------------------------------------------
constexpr int kTmaWarps = 5;
constexpr int kTmaRows = kReconRows;               // rows per item
constexpr int kTmaSeg = kReconSeg;                 // 16-byte vectors per row segment (2 KB)
constexpr int kTmaStages = 2;
constexpr long long kWaitCycles = 2000000000ll;    // ~1 s at 2 GHz

struct TmaSmem {
    uint4 ring[kTmaWarps][kTmaStages][kTmaRows * kTmaSeg];
    unsigned long long bar[kTmaWarps][kTmaStages];
    int item[kTmaWarps][kTmaStages];  // item whose first stage the slot holds; -1: no more items
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
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

// wait for the given phase parity, giving up after kWaitCycles
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitCycles) return false;
    return true;
}

__device__ __forceinline__ uint64_t evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, unsigned long long* bar,
                                         uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}

// stage geometry of chunk kc of a slice: n4 16-byte vectors per row, nst stages of kTmaSeg
// vectors (the last one shorter)
__device__ __forceinline__ void chunk_geom(const ReconLaunch& L, int kc, int& n4, int& nst) {
    const int epv = 16 / recon_esize(L.dtype);
    const int ncols = min(L.len - kc * L.kc, L.kc);
    n4 = (ncols + epv - 1) / epv;
    nst = (n4 + kTmaSeg - 1) / kTmaSeg;
}

// widening of packed elements: bfloat16 pairs are the upper halves of float32 words; an E4M3
// pair goes through an f16x2 conversion (exact), then each half to float32 (exact)
__device__ __forceinline__ float2 bf16x2_to_f32x2(uint32_t w) {
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}
__device__ __forceinline__ float4 e4m3x4_to_f32x4(uint32_t w) {
    float4 r;
    asm("{\n\t.reg .b16 lo, hi;\n\t.reg .b32 h01, h23;\n\t.reg .f16 a, b, c, d;\n\t"
        "mov.b32 {lo, hi}, %4;\n\t"
        "cvt.rn.f16x2.e4m3x2 h01, lo;\n\t"
        "cvt.rn.f16x2.e4m3x2 h23, hi;\n\t"
        "mov.b32 {a, b}, h01;\n\t"
        "mov.b32 {c, d}, h23;\n\t"
        "cvt.f32.f16 %0, a;\n\t"
        "cvt.f32.f16 %1, b;\n\t"
        "cvt.f32.f16 %2, c;\n\t"
        "cvt.f32.f16 %3, d;\n\t}"
        : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
        : "r"(w));
    return r;
}
// narrowing with round to nearest even (E4M3 saturating to +-448); element 0 in the low bits
__device__ __forceinline__ uint32_t f32x2_to_bf16x2(float x0, float x1) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(x1), "f"(x0));
    return d;
}
__device__ __forceinline__ uint32_t f32x4_to_e4m3x4(float x0, float x1, float x2, float x3) {
    uint32_t d;
    asm("{\n\t.reg .b16 lo, hi;\n\t"
        "cvt.rn.satfinite.e4m3x2.f32 lo, %2, %1;\n\t"
        "cvt.rn.satfinite.e4m3x2.f32 hi, %4, %3;\n\t"
        "mov.b32 %0, {lo, hi};\n\t}"
        : "=r"(d)
        : "f"(x0), "f"(x1), "f"(x2), "f"(x3));
    return d;
}

// one 16-byte vector of R times the matching slopes, into the two halves of acc
template <int DT>
__device__ __forceinline__ float2 vec_dot(uint4 r, const float4* sv, float2 acc) {
    if constexpr (DT == kReconF32) {
        return dot4x2(make_float4(__uint_as_float(r.x), __uint_as_float(r.y), __uint_as_float(r.z),
                                  __uint_as_float(r.w)),
                      sv[0], acc);
    } else if constexpr (DT == kReconBF16) {
        acc = ffma2(bf16x2_to_f32x2(r.x), make_float2(sv[0].x, sv[0].y), acc);
        acc = ffma2(bf16x2_to_f32x2(r.y), make_float2(sv[0].z, sv[0].w), acc);
        acc = ffma2(bf16x2_to_f32x2(r.z), make_float2(sv[1].x, sv[1].y), acc);
        return ffma2(bf16x2_to_f32x2(r.w), make_float2(sv[1].z, sv[1].w), acc);
    } else {
        const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) acc = dot4x2(e4m3x4_to_f32x4(w[i]), sv[i], acc);
        return acc;
    }
}

// Chunk geometry {n4, nst} of a full chunk and of the slice's last (possibly shorter) one,
// computed once per thread so that the per-stage path needs no division.
struct SliceGeom {
    int n_chunks;
    int full[2], last[2];
};

__device__ __forceinline__ SliceGeom slice_geom(const ReconLaunch& L) {
    SliceGeom g;
    g.n_chunks = (L.len + L.kc - 1) / L.kc;
    chunk_geom(L, 0, g.full[0], g.full[1]);
    chunk_geom(L, g.n_chunks - 1, g.last[0], g.last[1]);
    return g;
}

// One stage: the vectors e = lane + 32 j (j < 4) of the four rows.  A full stage (kTmaSeg
// vectors) needs no predicate; a short one guards loads and multiply-adds alike (registers of
// lanes past the end are never read).
template <bool FULL>
__device__ __forceinline__ void stage_load(const uint4* ring, int lane, int cnt, uint4 (&rv)[kTmaSeg / 32][kTmaRows]) {
    const int stride = FULL ? kTmaSeg : cnt;
#pragma unroll
    for (int j = 0; j < kTmaSeg / 32; ++j) {
        const int e = lane + 32 * j;
        if (FULL || e < cnt) {
#pragma unroll
            for (int q = 0; q < kTmaRows; ++q) rv[j][q] = ring[q * stride + e];
        }
    }
}

template <int DT, bool FULL>
__device__ __forceinline__ void stage_fma(const uint4 (&rv)[kTmaSeg / 32][kTmaRows], const float4 (&sv)[kTmaSeg / 32],
                                          const float4* s4, int e0, int lane, int cnt, float2 (&acc)[kTmaRows]) {
    constexpr int SPV = 4 / recon_esize(DT);
#pragma unroll
    for (int j = 0; j < kTmaSeg / 32; ++j) {
        const int e = lane + 32 * j;
        if (FULL || e < cnt) {
            float4 sj[SPV];
            if constexpr (DT == kReconF32) {
                sj[0] = sv[j];
            } else {
#pragma unroll
                for (int i = 0; i < SPV; ++i) sj[i] = __ldg(s4 + (e0 + e) * SPV + i);
            }
#pragma unroll
            for (int q = 0; q < kTmaRows; ++q) acc[q] = vec_dot<DT>(rv[j][q], sj, acc[q]);
        }
    }
}

// c += g sum_k partial[k][row] for one row: eight lanes per row (m = 0..7, consecutive lanes of
// one warp), lane m adds slots m, m + 8, ... (all its loads in flight at once), then a fixed
// shuffle tree; deterministic.  With the second-order controller:
// c_{k+1} = a1 c_k + a2 c_{k-1} + b0 dc_k + b1 dc_{k-1}.  Without partials the update is read
// from dc_in (batched product).  Every lane of the warp must call it.
__device__ __forceinline__ void reduce_row(const ReduceLaunch& L, long long row, int m, long long n_rows) {
    float a = 0.0f;
    if (row < n_rows) {
        if (L.partial) {
#pragma unroll 4
            for (int k = m; k < L.n_chunks; k += 8) a += __ldcg(L.partial + (size_t)k * L.n_cmd + row);
        } else if (m == 0) {
            a = L.dc_in[row];
        }
    }
    a += __shfl_xor_sync(0xffffffffu, a, 4);
    a += __shfl_xor_sync(0xffffffffu, a, 2);
    a += __shfl_xor_sync(0xffffffffu, a, 1);
    if (m == 0 && row < n_rows) {
        if (!L.use_ctl) {
            L.c[row] = fmaf(L.gain, a, L.c[row]);
        } else {
            const float c0 = L.c[row];
            float cn = L.a1 * c0;
            cn = fmaf(L.a2, L.c_prev[row], cn);
            cn = fmaf(L.b0, a, cn);
            cn = fmaf(L.b1, L.dc_prev[row], cn);
            L.c_prev[row] = c0;
            L.dc_prev[row] = a;
            L.c[row] = cn;
        }
    }
}

// Work items i = kc * n_rq + rq (row quad rq, chunk kc) are handed out one at a time by the
// slice's counter (zero when the step starts), so blocks that become resident late -- the
// sensing kernels share the SMs -- take only what is left.  Lane 0 of each warp is the producer:
// it claims items (one claim ahead, hiding the atomic's latency), records in the slot that
// receives an item's first stage which item it is (-1 once the counter is exhausted) and issues
// the copies.  The other lanes follow the slots in order.  Per stage: wait for the slot's copy,
// pull the stage into registers, let lane 0 refill the slot, then do the multiply-adds -- a slot
// is held only for its shared-memory loads, which keeps the warp's copies in flight.
template <int DT>
__global__ void __launch_bounds__(kTmaWarps * 32) recon_tma_kernel(ReconLaunch L) {
    constexpr int SPV = 4 / recon_esize(DT);   // float4 of slopes per 16-byte vector of R
    extern __shared__ __align__(128) unsigned char tma_raw[];
    TmaSmem& sm = *reinterpret_cast<TmaSmem*>(tma_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int st = 0; st < kTmaStages; ++st) mbar_init(&sm.bar[warp][st], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();
    const uint64_t pol = evict_first_policy();
    const int n_rq = L.n_rq;
    const SliceGeom g = slice_geom(L);
    const int n_items = n_rq * g.n_chunks;
    const uint4* R4 = reinterpret_cast<const uint4*>(L.R + L.base);
    const long long blk4 = (long long)kTmaRows * L.kc / (16 / recon_esize(DT));   // vectors per item block

    // producer state (used by lane 0 only)
    int p_next = 0, p_t = 0, p_n4 = 0, p_nst = 1, issued = 0;
    bool p_done = false;
    const uint4* p_src = R4;
    if (lane == 0) p_next = (int)atomicAdd(L.work, 1u);
    auto issue_next = [&](int st) {
        if (p_t == 0) {
            const int it = p_next;
            if (it >= n_items) {
                sm.item[warp][st] = -1;
                p_done = true;
                return;
            }
            p_next = (int)atomicAdd(L.work, 1u);
            const int kc = it / n_rq, rq = it - kc * n_rq;
            const int* q = kc == g.n_chunks - 1 ? g.last : g.full;
            p_n4 = q[0];
            p_nst = q[1];
            p_src = R4 + ((long long)kc * n_rq + rq) * blk4;
            sm.item[warp][st] = it;
        }
        const int cnt = min(kTmaSeg, p_n4 - p_t * kTmaSeg);
        const uint32_t bytes = (uint32_t)(kTmaRows * cnt) * 16u;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(&sm.bar[warp][st], bytes);
        bulk_g2s(sm.ring[warp][st], p_src + (long long)kTmaRows * kTmaSeg * p_t, bytes, &sm.bar[warp][st], pol);
        ++issued;
        if (++p_t == p_nst) p_t = 0;
    };
    if (lane == 0)
        for (int st = 0; st < kTmaStages && !p_done; ++st) issue_next(st);

    uint32_t parity = 0;  // bit st: parity of the next completion of slot st
    int consumed = 0;
    for (;;) {
        int it = 0;
        if (lane == 0) it = sm.item[warp][consumed % kTmaStages];
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it < 0) break;
        const int kc = it / n_rq, rq = it - kc * n_rq;
        const int* cg = kc == g.n_chunks - 1 ? g.last : g.full;
        const int n4 = cg[0], nst = cg[1];
        const float4* s4 = reinterpret_cast<const float4*>(L.s + L.col0 + kc * L.kc);
        float2 acc2[kTmaRows];
#pragma unroll
        for (int q = 0; q < kTmaRows; ++q) acc2[q] = make_float2(0.0f, 0.0f);
        for (int t = 0; t < nst; ++t, ++consumed) {
            const int st = consumed % kTmaStages;
            const int e0 = t * kTmaSeg, cnt = min(kTmaSeg, n4 - e0);
            const bool full = cnt == kTmaSeg;
            float4 sv[kTmaSeg / 32];
            if constexpr (DT == kReconF32) {
                // float32: the slopes of all four vectors are loaded before the wait
#pragma unroll
                for (int j = 0; j < kTmaSeg / 32; ++j) {
                    const int e = lane + 32 * j;
                    if (full || e < cnt) sv[j] = __ldg(s4 + e0 + e);
                }
            }
            if (!mbar_wait_bounded(&sm.bar[warp][st], (parity >> st) & 1u)) {
                // record the failure, let the copies still in flight land (bounded), stop the warp
                if (lane == 0) {
                    atomicExch(L.err, kErrReconTimeout);
                    for (int k = consumed + 1; k < issued; ++k) {
                        const int s2 = k % kTmaStages;
                        mbar_wait_bounded(&sm.bar[warp][s2], (parity >> s2) & 1u);
                    }
                }
                __syncwarp();
                return;
            }
            parity ^= 1u << st;
            const uint4* ring = sm.ring[warp][st];
            uint4 rv[kTmaSeg / 32][kTmaRows];
            if (full) stage_load<true>(ring, lane, cnt, rv);
            else stage_load<false>(ring, lane, cnt, rv);
            __syncwarp();  // every lane has read the slot before it is refilled
            if (lane == 0 && !p_done) issue_next(st);
            if (full) stage_fma<DT, true>(rv, sv, s4, e0, lane, cnt, acc2);
            else stage_fma<DT, false>(rv, sv, s4, e0, lane, cnt, acc2);
        }
        float acc[kTmaRows];
#pragma unroll
        for (int q = 0; q < kTmaRows; ++q) acc[q] = acc2[q].x + acc2[q].y;
#pragma unroll
        for (int q = 0; q < kTmaRows; ++q) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
        }
        if (lane == 0) {
            float* out = L.partial + (size_t)(L.chunk0 + kc) * L.n_cmd;
            const int row0 = rq * kTmaRows;
#pragma unroll
            for (int q = 0; q < kTmaRows; ++q)
                if (row0 + q < L.n_cmd) out[row0 + q] = DT == kReconE4M3 ? acc[q] * L.scale[row0 + q] : acc[q];
        }
    }
}

// 16 consecutive float32 elements of row r from column c (zero at and beyond column c_end)
__device__ __forceinline__ void load16(const float* row, int c, int c_end, float* x, int n) {
    for (int i = 0; i < n; ++i) x[i] = (c + i < c_end) ? row[c + i] : 0.0f;
}

// one 16-byte vector of codes from n = 16 / esize float32 elements
__device__ __forceinline__ uint4 encode_vec(int dtype, const float* x, float scale) {
    uint4 v;
    if (dtype == kReconF32) {
        v = make_uint4(__float_as_uint(x[0]), __float_as_uint(x[1]), __float_as_uint(x[2]), __float_as_uint(x[3]));
    } else if (dtype == kReconBF16) {
        v = make_uint4(f32x2_to_bf16x2(x[0], x[1]), f32x2_to_bf16x2(x[2], x[3]), f32x2_to_bf16x2(x[4], x[5]),
                       f32x2_to_bf16x2(x[6], x[7]));
    } else {
        float y[16];
        for (int i = 0; i < 16; ++i) y[i] = __fdiv_rn(x[i], scale);
        v = make_uint4(f32x4_to_e4m3x4(y[0], y[1], y[2], y[3]), f32x4_to_e4m3x4(y[4], y[5], y[6], y[7]),
                       f32x4_to_e4m3x4(y[8], y[9], y[10], y[11]), f32x4_to_e4m3x4(y[12], y[13], y[14], y[15]));
    }
    return v;
}

// Re-tiling: one thread per 16-byte vector of the slice (rows x chunk vectors); columns at or
// beyond the slice's end are stored as zeros.
__global__ void recon_tile_kernel(const float* __restrict__ src, long long ld, ReconLaunch L) {
    const int epv = 16 / recon_esize(L.dtype);
    const int kcv = L.kc / epv;
    const int n_chunks = (L.len + L.kc - 1) / L.kc;
    const long long nv_slice = (long long)kcv * n_chunks;
    const long long total = (long long)L.n_rq * kTmaRows * nv_slice;
    float x[16];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / nv_slice;
        const int cv = (int)(i - r * nv_slice);           // vector column inside the slice
        const int kc = cv / kcv, e4 = cv - kc * kcv;
        int n4, nst;
        chunk_geom(L, kc, n4, nst);
        if (e4 >= n4) continue;                            // padding of a short last chunk
        const float* row = src + r * ld + L.col0;
        load16(row, kc * L.kc + e4 * epv, L.len, x, epv);
        const float sc = (L.dtype == kReconE4M3) ? L.scale[r] : 1.0f;
        const int t = e4 / kTmaSeg, e = e4 - t * kTmaSeg;
        const int cnt = min(kTmaSeg, n4 - t * kTmaSeg);
        const int rq = (int)(r / kTmaRows), q = (int)(r % kTmaRows);
        uint4* dst = reinterpret_cast<uint4*>(const_cast<unsigned char*>(L.R) + L.base) +
                     ((long long)kc * L.n_rq + rq) * (long long)kTmaRows * kcv + (long long)kTmaRows * kTmaSeg * t +
                     q * cnt + e;
        *dst = encode_vec(L.dtype, x, sc);
    }
}

// per-row scale for E4M3: fl(max |R_r.| / 448), 1 for an all-zero row and for a row whose
// fl(max / 448) is below the smallest normal float 2^-126 (there every entry is below 448 2^-126
// and encodes to zero; a scale that underflowed to 0 would make 0 / 0 codes)
__global__ void recon_scale_kernel(const float* __restrict__ src, int cols, int ld, float* scale) {
    const long long r = blockIdx.x;
    float m = 0.0f;
    for (int j = threadIdx.x; j < cols; j += blockDim.x) m = fmaxf(m, fabsf(src[r * ld + j]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a = fmaxf(a, red[w]);
        const float sc = __fdiv_rn(a, 448.0f);
        scale[r] = sc >= 1.17549435e-38f ? sc : 1.0f;
    }
}

// row-major codes [rows][cols]: one thread per 16-byte vector of codes (cols a multiple of the
// vector's element count, checked by the caller) 
__global__ void quantize_rows_kernel(const float* __restrict__ src, int rows, int cols, int ld, int dtype,
                                     uint4* out, const float* scale) {
    const int epv = 16 / recon_esize(dtype);
    const int vpr = cols / epv;
    const long long total = (long long)rows * vpr;
    float x[16];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / vpr;
        const int v = (int)(i - r * vpr);
        load16(src + r * ld, v * epv, cols, x, epv);
        out[i] = encode_vec(dtype, x, dtype == kReconE4M3 ? scale[r] : 1.0f);
    }
}

// the update as a kernel of its own: eight lanes per row (reduce_row); the step counter
__global__ void recon_reduce_kernel(ReduceLaunch L) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0 && L.st) L.st->k_next = L.st->k + 1;
    const long long n_rows = (long long)L.n_cmd * (L.partial ? 1 : L.n_real);
    reduce_row(L, t >> 3, (int)(t & 7), n_rows);
}

// transpose of a row-major float32 [rows][cols] into [cols][ld_out] (float32 or bfloat16),
// 32 x 32 tiles through shared memory
template <bool BF16>
__global__ void transpose_kernel(const float* __restrict__ src, int rows, int cols, void* out, int ld_out) {
    __shared__ float tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        tile[i][threadIdx.x] = (r < rows && c < cols) ? src[(long long)r * cols + c] : 0.0f;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (c < cols && r < ld_out) {
            const float v = tile[threadIdx.x][i];
            if (BF16) {
                uint32_t h = f32x2_to_bf16x2(v, 0.0f) & 0xffffu;
                reinterpret_cast<uint16_t*>(out)[(long long)c * ld_out + r] = (uint16_t)h;
            } else {
                reinterpret_cast<float*>(out)[(long long)c * ld_out + r] = v;
            }
        }
    }
}

}  // namespace

cudaError_t launch_transpose(const float* src, int rows, int cols, void* out, int ld_out, int bf16, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((ld_out + 31) / 32)), block(32, 8);
    if (bf16) transpose_kernel<true><<<grid, block, 0, st>>>(src, rows, cols, out, ld_out);
    else transpose_kernel<false><<<grid, block, 0, st>>>(src, rows, cols, out, ld_out);
    return cudaGetLastError();
}

long long recon_slice_bytes(int n_rq, int len, int kc, int dtype) {
    const long long chunks = (len + kc - 1) / kc;
    return chunks * n_rq * (long long)kTmaRows * kc * recon_esize(dtype);
}

namespace {

// Self-check of the bounded waits: one thread waits on an mbarrier that nothing arrives at (its
// first phase never completes); the wait must give up after kWaitCycles and report, exactly as
// a product warp would, and the block then exits normally.
__global__ void wait_probe_kernel(int* err) {
    __shared__ unsigned long long bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0u)) atomicExch(err, kErrReconTimeout);
}

}  // namespace

cudaError_t launch_wait_probe(int* err, cudaStream_t s) {
    wait_probe_kernel<<<1, 32, 0, s>>>(err);
    return cudaGetLastError();
}

cudaError_t recon_prepare() {
    cudaError_t e = cudaFuncSetAttribute(recon_tma_kernel<kReconF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(TmaSmem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(recon_tma_kernel<kReconBF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(TmaSmem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(recon_tma_kernel<kReconE4M3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(TmaSmem));
    return e;
}

cudaError_t launch_recon(const ReconLaunch& L, cudaStream_t s) {
    if (L.n_cmd <= 0 || L.len <= 0) return cudaSuccess;
    if (!L.work) return cudaErrorInvalidValue;
    const int n_items = L.n_rq * ((L.len + L.kc - 1) / L.kc);
    const int need = (n_items + kTmaWarps - 1) / kTmaWarps;
    int ctas = (L.max_ctas > 0 && L.max_ctas < need) ? L.max_ctas : need;
    if (L.dtype == kReconF32) recon_tma_kernel<kReconF32><<<(unsigned)ctas, kTmaWarps * 32, sizeof(TmaSmem), s>>>(L);
    else if (L.dtype == kReconBF16) recon_tma_kernel<kReconBF16><<<(unsigned)ctas, kTmaWarps * 32, sizeof(TmaSmem), s>>>(L);
    else if (L.dtype == kReconE4M3) recon_tma_kernel<kReconE4M3><<<(unsigned)ctas, kTmaWarps * 32, sizeof(TmaSmem), s>>>(L);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_recon_scales(const float* src, int rows, int cols, int ld, float* scale, cudaStream_t s) {
    if (rows <= 0) return cudaSuccess;
    recon_scale_kernel<<<(unsigned)rows, 256, 0, s>>>(src, cols, ld, scale);
    return cudaGetLastError();
}

cudaError_t launch_quantize_rows(const float* src, int rows, int cols, int ld, int dtype, void* out,
                                 const float* scale, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    quantize_rows_kernel<<<2048, 256, 0, s>>>(src, rows, cols, ld, dtype, reinterpret_cast<uint4*>(out), scale);
    return cudaGetLastError();
}

cudaError_t launch_recon_tile(const float* src, int ld, const ReconLaunch& L, cudaStream_t s) {
    if (L.len <= 0) return cudaSuccess;
    recon_tile_kernel<<<2048, 256, 0, s>>>(src, ld, L);
    return cudaGetLastError();
}

cudaError_t launch_recon_reduce(const ReduceLaunch& L, cudaStream_t s) {
    const long long rows = (long long)(L.n_cmd > 0 ? L.n_cmd : 1) * (L.partial ? 1 : (L.n_real > 0 ? L.n_real : 1));
    const long long n = 8LL * rows;
    recon_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(L);
    return cudaGetLastError();
}

}  // namespace mcao
