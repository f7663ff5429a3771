// DM surfaces (Gaussian influence functions, "Influence function and modal base" of
// arXiv:1608.00386): S = sum_j c_j exp(-|x - x_j|^2 / 2 sigma^2), with exp(-pitch^2/2 sigma^2)
// equal to the coupling.  The Gaussian factorises, so S = Gy C Gx^T exactly.
//  pass 1: T = C Gx^T, one block per actuator row and 256 surface columns, the command row
//          gathered once into shared memory; each Gx row is restricted to the actuators whose
//          weight is at least 1e-10 (dropped terms are below float rounding of the surface).
//  pass 2: S = Gy T by 32 x 32 output tiles; the tile's Gy rows and T columns over the union of
//          its rows' bands are staged in shared memory, each thread forms four outputs.
#include "mcao_internal.h"

namespace mcao {

namespace {

constexpr int kTile = 32;
constexpr int kMaxBand = 64;   // union band of a 32-row tile (checked on the host)
constexpr int kMaxAct = kDmMaxAct;

__global__ void __launch_bounds__(256) dm_pass1(DmLaunch L) {
    __shared__ float s_c[kMaxAct];
    if (blockIdx.x == 0 && threadIdx.x == 0 && L.st) L.st->k = L.st->k_next;
    // block -> (dm, actuator row b, column block)
    int blk = blockIdx.x;
    int m = 0;
    const DmDesc* d = nullptr;
    int per = 0;
    for (; m < L.n_dm; ++m) {
        d = &L.desc[m];
        per = d->ny * ((d->surf_n + 255) / 256);
        if (blk < per) break;
        blk -= per;
    }
    if (m >= L.n_dm) return;
    const int cb = (d->surf_n + 255) / 256;
    const int b = blk / cb, i = (blk % cb) * 256 + threadIdx.x;
    const int* map = L.act_map + d->map_off + (long long)b * d->nx;
    for (int a = threadIdx.x; a < d->nx; a += blockDim.x) {
        int q = map[a];
        s_c[a] = (q >= 0) ? L.c[q] : 0.0f;
    }
    __syncthreads();
    if (i >= d->surf_n) return;
    const int2 band = L.band[d->band_off + i];
    const float* g = L.g + d->gx_off + (long long)i * d->nx;
    float acc = 0.0f;
    for (int a = band.x; a < band.y; ++a) acc = fmaf(__ldg(g + a), s_c[a], acc);
    L.tmp[d->tmp_off + (long long)b * d->surf_n + i] = acc;
}

__global__ void __launch_bounds__(256) dm_pass2(DmLaunch L) {
    __shared__ float s_T[kMaxBand][kTile];
    __shared__ float s_G[kTile][kMaxBand + 1];
    int t = blockIdx.x;
    int m = 0;
    while (m + 1 < L.n_dm && t >= L.tile_start[m + 1]) ++m;
    const DmDesc& d = L.desc[m];
    t -= L.tile_start[m];
    const int n = d.surf_n;
    const int j0 = (t / d.tiles_x) * kTile, i0 = (t % d.tiles_x) * kTile;
    const int2 tb = L.band[d.tband_off + j0 / kTile];
    const int b_lo = tb.x;
    const int nb = tb.y - tb.x;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int c0 = 0; c0 < nb; c0 += kMaxBand) {
        const int cn = min(kMaxBand, nb - c0);
        for (int q = threadIdx.x; q < cn * kTile; q += blockDim.x) {
            int bb = q / kTile, ii = q % kTile;
            int i = i0 + ii;
            s_T[bb][ii] = (i < n) ? L.tmp[d.tmp_off + (long long)(b_lo + c0 + bb) * n + i] : 0.0f;
        }
        for (int q = threadIdx.x; q < kTile * cn; q += blockDim.x) {
            int jj = q / cn, bb = q % cn;
            int j = j0 + jj;
            s_G[jj][bb] = (j < n) ? L.g[d.gy_off + (long long)j * d.ny + b_lo + c0 + bb] : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int jj = ty * 4 + r;
            float a = acc[r];
            for (int bb = 0; bb < cn; ++bb) a = fmaf(s_G[jj][bb], s_T[bb][tx], a);
            acc[r] = a;
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int j = j0 + ty * 4 + r, i = i0 + tx;
        if (j < n && i < n) L.surf[d.surf_off + (long long)j * n + i] = acc[r];
    }
}

__global__ void begin_step_kernel(StepState* st) {
    if (threadIdx.x == 0 && blockIdx.x == 0) st->k = st->k_next;
}

}  // namespace

cudaError_t launch_dm_surfaces(const DmLaunch& L, cudaStream_t s) {
    if (L.n_dm <= 0) return launch_begin_step(L.st, s);
    dm_pass1<<<(unsigned)L.pass1_blocks, 256, 0, s>>>(L);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dm_pass2<<<(unsigned)L.tile_start[L.n_dm], 256, 0, s>>>(L);
    return cudaGetLastError();
}

cudaError_t launch_begin_step(StepState* st, cudaStream_t s) {
    if (!st) return cudaSuccess;
    begin_step_kernel<<<1, 32, 0, s>>>(st);
    return cudaGetLastError();
}

}  // namespace mcao
