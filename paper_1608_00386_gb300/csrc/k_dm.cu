// DM surfaces (Gaussian influence functions, "Influence function and modal base" of
// arXiv:1608.00386): S = sum_j c_j exp(-|x - x_j|^2 / 2 sigma^2), with exp(-pitch^2/2 sigma^2)
// equal to the coupling.  The Gaussian factorises, so S = Gy C Gx^T exactly; each row of Gx
// and Gy is restricted to the actuators whose weight is at least 1e-10 (dropped terms are
// below float rounding of the surface).
#include "mcao_internal.h"

namespace mcao {

namespace {

__device__ __forceinline__ int find_dm(long long t, const long long* start, int n) {
    int m = 0;
    while (m + 1 < n && t >= start[m + 1]) ++m;
    return m;
}

// T[b][i] = sum_{a in band_x(i)} Gx[i][a] C[b][a], C[b][a] = c[map[b][a]] (0 if invalid)
__global__ void dm_pass1(DmLaunch L) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0 && L.st) L.st->k = L.st->k_next;
    if (t >= L.tmp_total) return;
    int m = find_dm(t, L.tmp_start, L.n_dm);
    const DmDesc d = L.desc[m];
    long long local = t - L.tmp_start[m];
    int b = (int)(local / d.surf_n), i = (int)(local % d.surf_n);
    int2 band = L.band[d.band_off + i];
    const float* g = L.g + d.gx_off + (long long)i * d.nx;
    const int* map = L.act_map + d.map_off + (long long)b * d.nx;
    float acc = 0.0f;
    for (int a = band.x; a < band.y; ++a) {
        int q = map[a];
        if (q >= 0) acc = fmaf(g[a], L.c[q], acc);
    }
    L.tmp[d.tmp_off + (long long)b * d.surf_n + i] = acc;
}

// S[j][i] = sum_{b in band_y(j)} Gy[j][b] T[b][i]
__global__ void dm_pass2(DmLaunch L) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= L.surf_total) return;
    int m = find_dm(t, L.surf_start, L.n_dm);
    const DmDesc d = L.desc[m];
    long long local = t - L.surf_start[m];
    int j = (int)(local / d.surf_n), i = (int)(local % d.surf_n);
    int2 band = L.band[d.band_off + d.surf_n + j];
    const float* g = L.g + d.gy_off + (long long)j * d.ny;
    const float* T = L.tmp + d.tmp_off + i;
    float acc = 0.0f;
    for (int b = band.x; b < band.y; ++b) acc = fmaf(g[b], T[(long long)b * d.surf_n], acc);
    L.surf[d.surf_off + (long long)j * d.surf_n + i] = acc;
}

__global__ void begin_step_kernel(StepState* st) {
    if (threadIdx.x == 0 && blockIdx.x == 0) st->k = st->k_next;
}

}  // namespace

cudaError_t launch_dm_surfaces(const DmLaunch& L, cudaStream_t s) {
    if (L.n_dm <= 0) return launch_begin_step(L.st, s);
    const int threads = 256;
    long long b1 = (L.tmp_total + threads - 1) / threads;
    dm_pass1<<<(unsigned)(b1 > 0 ? b1 : 1), threads, 0, s>>>(L);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    long long b2 = (L.surf_total + threads - 1) / threads;
    if (b2 > 0) dm_pass2<<<(unsigned)b2, threads, 0, s>>>(L);
    return cudaGetLastError();
}

cudaError_t launch_begin_step(StepState* st, cudaStream_t s) {
    if (!st) return cudaSuccess;
    begin_step_kernel<<<1, 32, 0, s>>>(st);
    return cudaGetLastError();
}

}  // namespace mcao
