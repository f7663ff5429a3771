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
// Streaming.  At most one block per SM (3 warps).  Each warp owns a four-stage ring in
// shared memory and keeps it filled with TMA bulk copies (cp.async.bulk, completion counted on a
// per-stage mbarrier, L2 evict-first policy).  R is held stage-tiled (see ReconLaunch), so each
// stage -- four row segments of up to 2 KB -- is one contiguous copy of up to 8 KB (bulk copies
// that small lose bandwidth), and up to 96 KB per SM are in flight.  The block needs
// few registers and warps, which leaves each SM room for three wavefront-sensor blocks that run
// concurrently, hiding their ALU work under the HBM stream.  Every mbarrier wait is bounded
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
constexpr int kTmaWarps = 3;
constexpr int kTmaRows = kReconRows;               // rows per item
constexpr int kTmaSeg = kReconSeg;                 // float4 per row segment (2 KB)
constexpr int kTmaStages = 4;
constexpr long long kWaitCycles = 2000000000ll;    // ~1 s at 2 GHz

struct TmaSmem {
    float4 ring[kTmaWarps][kTmaStages][kTmaRows * kTmaSeg];
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

// stage geometry of chunk kc of a slice: n4 float4 per row, nst stages of seg float4
__device__ __forceinline__ void chunk_geom(const ReconLaunch& L, int kc, int& n4, int& nst, int& seg) {
    const int ncols = min(L.len - kc * L.kc, L.kc);
    n4 = (ncols + 3) / 4;
    nst = (n4 + kTmaSeg - 1) / kTmaSeg;
    seg = (n4 + nst - 1) / nst;
}

// Chunk geometry {n4, nst, seg} of a full chunk and of the slice's last (possibly shorter) one,
// computed once per thread so that the per-stage path needs no division.
struct SliceGeom {
    int n_chunks;
    int full[3], last[3];
};

__device__ __forceinline__ SliceGeom slice_geom(const ReconLaunch& L) {
    SliceGeom g;
    g.n_chunks = (L.len + L.kc - 1) / L.kc;
    chunk_geom(L, 0, g.full[0], g.full[1], g.full[2]);
    chunk_geom(L, g.n_chunks - 1, g.last[0], g.last[1], g.last[2]);
    return g;
}

// Work items i = kc * n_rq + rq (row quad rq, chunk kc) are handed out one at a time by the
// slice's counter (zero when the step starts), so blocks that become resident late -- the
// sensing kernels share the SMs -- take only what is left.  Lane 0 of each warp is the producer:
// it claims items (one claim ahead, hiding the atomic's latency), records in the slot that
// receives an item's first stage which item it is (-1 once the counter is exhausted) and issues
// the copies.  The other lanes follow the slots in order.  Per stage: wait for the slot's copy,
// pull the stage into registers, let lane 0 refill the slot, then do the multiply-adds -- a slot
// is held only for its shared-memory loads, which keeps four copies per warp in flight.
__global__ void __launch_bounds__(kTmaWarps * 32) recon_tma_kernel(ReconLaunch L) {
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
    const float4* R4 = reinterpret_cast<const float4*>(L.R + L.base);
    const long long blk4 = (long long)L.kc;   // float4 per item block: 4 rows x kc floats / 4

    // producer state (used by lane 0 only)
    int p_next = 0, p_t = 0, p_n4 = 0, p_nst = 1, p_seg = 1, issued = 0;
    bool p_done = false;
    const float4* p_src = R4;
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
            p_seg = q[2];
            p_src = R4 + ((long long)kc * n_rq + rq) * blk4;
            sm.item[warp][st] = it;
        }
        const int cnt = min(p_seg, p_n4 - p_t * p_seg);
        const uint32_t bytes = (uint32_t)(kTmaRows * cnt) * 16u;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(&sm.bar[warp][st], bytes);
        bulk_g2s(sm.ring[warp][st], p_src + (long long)kTmaRows * p_seg * p_t, bytes, &sm.bar[warp][st], pol);
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
        const int n4 = cg[0], nst = cg[1], seg = cg[2];
        const float4* s4 = reinterpret_cast<const float4*>(L.s + L.col0 + kc * L.kc);
        float2 acc2[kTmaRows];
#pragma unroll
        for (int q = 0; q < kTmaRows; ++q) acc2[q] = make_float2(0.0f, 0.0f);
        for (int t = 0; t < nst; ++t, ++consumed) {
            const int st = consumed % kTmaStages;
            const int e0 = t * seg, cnt = min(seg, n4 - e0);
            float4 sv[kTmaSeg / 32];
#pragma unroll
            for (int j = 0; j < kTmaSeg / 32; ++j) {
                const int e = lane + 32 * j;
                sv[j] = e < cnt ? __ldg(s4 + e0 + e) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
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
            const float4* ring = sm.ring[warp][st];
            float4 rv[kTmaSeg / 32][kTmaRows];
#pragma unroll
            for (int j = 0; j < kTmaSeg / 32; ++j) {
                const int e = lane + 32 * j;
#pragma unroll
                for (int q = 0; q < kTmaRows; ++q)
                    rv[j][q] = e < cnt ? ring[q * cnt + e] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
            __syncwarp();  // every lane has read the slot before it is refilled
            if (lane == 0 && !p_done) issue_next(st);
#pragma unroll
            for (int j = 0; j < kTmaSeg / 32; ++j)
#pragma unroll
                for (int q = 0; q < kTmaRows; ++q) acc2[q] = dot4x2(rv[j][q], sv[j], acc2[q]);
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
                if (row0 + q < L.n_cmd) out[row0 + q] = acc[q];
        }
    }
}

// Re-tiling: one thread per float4 of the slice in the source layout (rows x chunk columns).
__global__ void recon_tile_kernel(const float4* __restrict__ src, long long ld4, ReconLaunch L) {
    const long long n4_slice = (long long)(L.kc / 4) * ((L.len + L.kc - 1) / L.kc);
    const long long total = (long long)L.n_rq * kTmaRows * n4_slice;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / n4_slice;
        const int c4 = (int)(i - r * n4_slice);           // float4 column inside the slice
        const int kc = c4 / (L.kc / 4), e4 = c4 - kc * (L.kc / 4);
        int n4, nst, seg;
        chunk_geom(L, kc, n4, nst, seg);
        float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (e4 < n4) v = src[r * ld4 + L.col0 / 4 + c4];
        else continue;                                     // padding of a short last chunk
        const int t = e4 / seg, e = e4 - t * seg;
        const int cnt = min(seg, n4 - t * seg);
        const int rq = (int)(r / kTmaRows), q = (int)(r % kTmaRows);
        float4* dst = reinterpret_cast<float4*>(const_cast<float*>(L.R) + L.base) +
                      ((long long)kc * L.n_rq + rq) * (long long)L.kc + (long long)kTmaRows * seg * t + q * cnt + e;
        *dst = v;
    }
}

__global__ void recon_reduce_kernel(ReduceLaunch L) {
    int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row == 0 && L.st) L.st->k_next = L.st->k + 1;
    if (row >= L.n_cmd) return;
    float acc = 0.0f;
    for (int kc = 0; kc < L.n_chunks; ++kc) acc += L.partial[(size_t)kc * L.n_cmd + row];
    L.c[row] = fmaf(L.gain, acc, L.c[row]);
}

}  // namespace

long long recon_slice_floats(int n_rq, int len, int kc) {
    const long long chunks = (len + kc - 1) / kc;
    return chunks * n_rq * (long long)kTmaRows * kc;
}

cudaError_t recon_prepare() {
    return cudaFuncSetAttribute(recon_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TmaSmem));
}

cudaError_t launch_recon(const ReconLaunch& L, cudaStream_t s) {
    if (L.n_cmd <= 0 || L.len <= 0) return cudaSuccess;
    if (!L.work) return cudaErrorInvalidValue;
    const int n_items = L.n_rq * ((L.len + L.kc - 1) / L.kc);
    const int need = (n_items + kTmaWarps - 1) / kTmaWarps;
    int ctas = (L.max_ctas > 0 && L.max_ctas < need) ? L.max_ctas : need;
    recon_tma_kernel<<<(unsigned)ctas, kTmaWarps * 32, sizeof(TmaSmem), s>>>(L);
    return cudaGetLastError();
}

cudaError_t launch_recon_tile(const float* src, int ld, const ReconLaunch& L, cudaStream_t s) {
    if (L.len <= 0) return cudaSuccess;
    recon_tile_kernel<<<2048, 256, 0, s>>>(reinterpret_cast<const float4*>(src), ld / 4, L);
    return cudaGetLastError();
}

cudaError_t launch_recon_reduce(const ReduceLaunch& L, cudaStream_t s) {
    int n = L.n_cmd > 0 ? L.n_cmd : 1;
    recon_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(L);
    return cudaGetLastError();
}

}  // namespace mcao
