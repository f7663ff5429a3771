// DM surfaces (Gaussian influence functions, "Influence function and modal base" of
// arXiv:1608.00386): S = sum_j c_j exp(-|x - x_j|^2 / 2 sigma^2), with exp(-pitch^2/2 sigma^2)
// equal to the coupling.  The Gaussian factorises, so S = Gy C Gx^T exactly.  One block per
// 64 x 64 block of the surface (the whole step's DMs in one wave of blocks): the block's
// actuator sub-grid C (rows and columns whose weight on the block is at least 1e-10; dropped
// terms are below float rounding of the surface), the matching columns of Gx^T and Gy^T (tables
// stored transposed, so that these loads are contiguous) and T = C Gx^T are staged in shared
// memory, then S = Gy T with a 4 x 4 register tile per thread.  A translated or magnified DM has
// its transform folded into Gx and Gy; a rotated one evaluates every sample against the
// actuators around its position in the DM's own frame.
#include "mcao_internal.h"

namespace mcao {

namespace {

constexpr int kBk = kDmBlock;
constexpr int kDmThreads = 256;

// floats of the command sub-grid [nb][nb + 1], rounded up so that the tables after it stay
// 16-byte aligned
__host__ __device__ __forceinline__ int dm_c_floats(int nb) { return (nb * (nb + 1) + 3) / 4 * 4; }

// actuator band [lo, hi) of block t along one axis: the union of its two tiles' bands
__device__ __forceinline__ int2 block_band(const int2* band, long long off, int t, int tiles) {
    const int2 a = band[off + 2 * t];
    const int2 b = (2 * t + 1 < tiles) ? band[off + 2 * t + 1] : make_int2(0, 0);
    if (a.y <= a.x) return b;
    if (b.y <= b.x) return a;
    return make_int2(min(a.x, b.x), max(a.y, b.y));
}

__global__ void __launch_bounds__(kDmThreads, 3) dm_surface_kernel(DmLaunch L) {
    extern __shared__ __align__(16) float dm_sm[];
    if (blockIdx.x == 0 && blockIdx.y == 0) {
        if (threadIdx.x == 0 && L.st) L.st->k = L.st->k_next;
        for (int i = threadIdx.x; i < L.n_work; i += blockDim.x) L.work[i] = 0u;
    }
    const int real = blockIdx.y;   // realization
    const float* cmd = L.c + (long long)real * L.n_cmd;
    int t = blockIdx.x;
    int m = 0;
    while (m + 1 < L.n_dm && t >= L.tile_start[m + 1]) ++m;
    const DmDesc& d = L.desc[m];
    t -= L.tile_start[m];
    const int n = d.surf_n;
    const int nbx = (d.tiles_x + 1) / 2;
    const int by_i = t / nbx, bx_i = t - by_i * nbx;
    const int j0 = by_i * kBk, i0 = bx_i * kBk;
    float* surf = L.surf + real * L.surf_stride + d.surf_off;
    const int tid = threadIdx.x;
    if (d.general) {
        // rotated DM: each sample q = R(-rot)((x, y) - shift) / mag weighs the actuators within rc
        // pitches directly
        const float c0 = 0.5f * (float)(n - 1), ca = 0.5f * (float)(d.nx - 1), cb = 0.5f * (float)(d.ny - 1);
        for (int q = tid; q < kBk * kBk; q += kDmThreads) {
            const int i = i0 + (q & (kBk - 1)), j = j0 + q / kBk;
            if (i >= n || j >= n) continue;
            const float x = ((float)i - c0) * d.dx - d.shx, y = ((float)j - c0) * d.dx - d.shy;
            const float ua = (d.cr * x + d.sr * y) * d.inv_mag / d.pitch + ca;
            const float ub = (-d.sr * x + d.cr * y) * d.inv_mag / d.pitch + cb;
            const int a0 = max(0, (int)ceilf(ua - d.rc)), a1 = min(d.nx - 1, (int)floorf(ua + d.rc));
            const int b0 = max(0, (int)ceilf(ub - d.rc)), b1 = min(d.ny - 1, (int)floorf(ub + d.rc));
            float acc = 0.0f;
            for (int b = b0; b <= b1; ++b) {
                const float dy = (ub - (float)b) * d.pitch;
                float row = 0.0f;
                for (int a = a0; a <= a1; ++a) {
                    const int idx = L.act_map[d.map_off + (long long)b * d.nx + a];
                    if (idx < 0) continue;
                    const float dxa = (ua - (float)a) * d.pitch;
                    row = fmaf(cmd[idx], expf(-dxa * dxa * d.inv2s2), row);
                }
                acc = fmaf(expf(-dy * dy * d.inv2s2), row, acc);
            }
            surf[(long long)j * n + i] = acc;
        }
        return;
    }
    const int2 bx = block_band(L.band, d.tband_x, bx_i, d.tiles_x);
    const int2 by = block_band(L.band, d.tband_y, by_i, d.tiles_x);
    const int na = bx.y - bx.x, nb = by.y - by.x;
    const int NB = L.nb, ldc = NB + 1;
    float* sC = dm_sm;                        // [nb][ldc]     commands of the band
    float* sGx = dm_sm + dm_c_floats(NB);     // [na][64]      Gx^T: actuator column, sample column
    float* sGy = sGx + NB * kBk;              // [nb][64]      Gy^T: actuator row, sample row
    float* sT = sGy + NB * kBk;               // [nb][64]      T = C Gx^T
    // Stage the commands (2-D thread mapping: no division by the runtime band sizes) and the
    // transposed weights of the block's 64 columns and 64 rows (zero beyond the surface).  Each
    // pass issues all of its loads before any store, so that the block waits for about one L2
    // round trip per pass instead of one per row: a pass covers 32 band rows of both tables, and
    // 32 x 32 commands (the bands of the configurations here fit in one pass).
    {
        constexpr int kRows = 32 / (kDmThreads / kBk);    // rows per thread and pass: 8
        const int s = tid & (kBk - 1), r0 = tid / kBk;
        const bool in_x = i0 + s < n, in_y = j0 + s < n;
        for (int rb = 0; rb < na || rb < nb; rb += 32) {
            float gx[kRows], gy[kRows];
#pragma unroll
            for (int k = 0; k < kRows; ++k) {
                const int r = rb + r0 + k * (kDmThreads / kBk);
                gx[k] = (r < na && in_x) ? __ldg(L.g + d.gxt_off + (long long)(bx.x + r) * n + i0 + s) : 0.0f;
                gy[k] = (r < nb && in_y) ? __ldg(L.g + d.gyt_off + (long long)(by.x + r) * n + j0 + s) : 0.0f;
            }
#pragma unroll
            for (int k = 0; k < kRows; ++k) {
                const int r = rb + r0 + k * (kDmThreads / kBk);
                if (r < na) sGx[r * kBk + s] = gx[k];
                if (r < nb) sGy[r * kBk + s] = gy[k];
            }
        }
        constexpr int kCmd = 32 / (kDmThreads / 32);      // command rows per thread and pass: 4
        const int lane = tid & 31, w = tid >> 5;
        for (int b0 = 0; b0 < nb; b0 += 32)
            for (int a0 = 0; a0 < na; a0 += 32) {
                const int aa = a0 + lane;
                int idx[kCmd];
#pragma unroll
                for (int k = 0; k < kCmd; ++k) {
                    const int bb = b0 + w + k * (kDmThreads / 32);
                    idx[k] = (bb < nb && aa < na) ? __ldg(L.act_map + d.map_off + (long long)(by.x + bb) * d.nx + bx.x + aa)
                                                  : -1;
                }
                float cv[kCmd];
#pragma unroll
                for (int k = 0; k < kCmd; ++k) cv[k] = idx[k] >= 0 ? cmd[idx[k]] : 0.0f;
#pragma unroll
                for (int k = 0; k < kCmd; ++k) {
                    const int bb = b0 + w + k * (kDmThreads / 32);
                    if (bb < nb && aa < na) sC[bb * ldc + aa] = cv[k];
                }
            }
    }
    __syncthreads();
    // T[bb][ii] = sum_aa C[bb][aa] Gx[ii][aa]: thread -> columns c4 .. c4 + 3 of rows bb
    const int c4 = (tid & 15) * 4;
    for (int bb = tid >> 4; bb < nb; bb += kDmThreads / 16) {
        float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        for (int aa = 0; aa < na; ++aa) {
            const float c = sC[bb * ldc + aa];
            const float4 g = *reinterpret_cast<const float4*>(sGx + aa * kBk + c4);
            acc.x = fmaf(c, g.x, acc.x);
            acc.y = fmaf(c, g.y, acc.y);
            acc.z = fmaf(c, g.z, acc.z);
            acc.w = fmaf(c, g.w, acc.w);
        }
        *reinterpret_cast<float4*>(sT + bb * kBk + c4) = acc;
    }
    __syncthreads();
    // S[jj][ii] = sum_bb Gy[jj][bb] T[bb][ii]: thread -> rows r4 .. r4 + 3, columns c4 .. c4 + 3
    const int r4 = (tid >> 4) * 4;
    float acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = 0.0f;
    for (int bb = 0; bb < nb; ++bb) {
        const float4 gy = *reinterpret_cast<const float4*>(sGy + bb * kBk + r4);
        const float4 tv = *reinterpret_cast<const float4*>(sT + bb * kBk + c4);
        const float g4[4] = {gy.x, gy.y, gy.z, gy.w}, t4[4] = {tv.x, tv.y, tv.z, tv.w};
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(g4[r], t4[c], acc[r][c]);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int j = j0 + r4 + r;
        if (j >= n) break;
        float* row = surf + (long long)j * n;
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (i0 + c4 + c < n) row[i0 + c4 + c] = acc[r][c];
    }
}

__global__ void begin_step_kernel(StepState* st, unsigned int* work, int n_work) {
    if (threadIdx.x == 0 && st) st->k = st->k_next;
    for (int i = threadIdx.x; i < n_work; i += blockDim.x) work[i] = 0u;
}

}  // namespace

size_t dm_smem_bytes(int nb) { return sizeof(float) * (size_t)(dm_c_floats(nb) + 3 * nb * kBk); }

cudaError_t dm_prepare() {
    // the attribute belongs to the kernel, not to one simulation: allow the largest block band
    // the host admits (two tiles of kDmMaxBand), so that simulations of different bands coexist
    return cudaFuncSetAttribute(dm_surface_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)dm_smem_bytes(2 * kDmMaxBand));
}

cudaError_t launch_dm_surfaces(const DmLaunch& L, cudaStream_t s) {
    if (L.n_dm <= 0) return launch_begin_step(L.st, L.work, L.n_work, s);
    dm_surface_kernel<<<dim3((unsigned)L.tile_start[L.n_dm], (unsigned)(L.n_real > 0 ? L.n_real : 1)), kDmThreads,
                        dm_smem_bytes(L.nb), s>>>(L);
    return cudaGetLastError();
}

cudaError_t launch_begin_step(StepState* st, unsigned int* work, int n_work, cudaStream_t s) {
    if (!st && n_work <= 0) return cudaSuccess;
    begin_step_kernel<<<1, 32, 0, s>>>(st, work, n_work);
    return cudaGetLastError();
}

}  // namespace mcao
