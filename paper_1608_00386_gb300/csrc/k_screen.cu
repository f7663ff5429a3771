// Phase screens on the GPU ("The atmospheric layers generation" of arXiv:1608.00386: phase
// screens of the turbulent layers from a turbulence spectrum).  The FFT method: on the discrete
// frequency grid of an n x n periodic screen of pitch `pixel`, complex Gaussian coefficients
// c = (z_c + i z_s) sqrt(PSD(kappa)) dk with the von Karman spectrum
// PSD = 0.023 r0^(-5/3) (kappa^2 + L0^-2)^(-11/6) (kappa in cycles per metre), c(0, 0) = 0,
// evaluated in float in units of the frequency cell dk = 1 / (n pixel):
// sqrt(PSD) dk = sqrt(0.023 r0^(-5/3)) (n pixel)^(5/6) (kx'^2 + ky'^2 + (n pixel / L0)^2)^(-11/12);
// the screen is Re sum_k c_k exp(+2 pi i k x / n) (an unnormalized inverse DFT), computed as
// the real part of the forward DFT of conj(c).  (z_c, z_s) is the Box-Muller pair of the
// detector-noise sampler drawn from Philox4x32-10 with counter (index, 0, 0, 1), key = seed.
// Two passes of row FFTs in shared memory, each storing its result transposed: the first
// generates its rows of coefficients in place (no coefficient array in HBM), the second keeps
// the real part.
#include "device_common.cuh"
#include "mcao_internal.h"

namespace mcao {

namespace {

constexpr int kScreenThreads = 512;
constexpr size_t kScreenSmemTarget = 113 * 1024;   // two blocks per SM

// rows per block: as many as fit two blocks per SM, 1..8
__host__ __device__ constexpr int screen_rows(int n) {
    return (int)((kScreenSmemTarget - sizeof(float2) * (size_t)n) / (2 * sizeof(float2) * (size_t)n)) < 1 ? 1
         : (int)((kScreenSmemTarget - sizeof(float2) * (size_t)n) / (2 * sizeof(float2) * (size_t)n)) > 8 ? 8
         : (int)((kScreenSmemTarget - sizeof(float2) * (size_t)n) / (2 * sizeof(float2) * (size_t)n));
}

__global__ void screen_twiddle_kernel(int n, float2* W) {
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(-2.0 * (double)m / (double)n, &s, &c);
        W[m] = make_float2((float)c, (float)s);
    }
}

// Twiddle table of the compile-time transform laid out stage by stage, so that a warp's
// butterflies (consecutive k) read consecutive entries: for the stage of sub-length ns and
// radix R, entry off + (r - 1) ns + k = exp(-2 pi i r k / (ns R)), r = 1 .. R-1, k < ns (the
// same float values as the single table exp(-2 pi i m / N) at m = r k N / (ns R)).
template <int N>
__global__ void screen_stage_twiddles(float2* T) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    int off = 0, ns = 1;
    while (ns < N) {
        const int R = ct_radix(N / ns);
        const int cnt = ns * (R - 1);
        if (e < off + cnt) {
            const int q = e - off, r = q / ns + 1, k = q - (r - 1) * ns;
            const int m = (r * k * (N / (ns * R))) % N;
            double sn, cs;
            sincospi(-2.0 * (double)m / (double)N, &sn, &cs);
            T[e] = make_float2((float)cs, (float)sn);
            return;
        }
        off += cnt;
        ns *= R;
    }
}

struct ScreenPass {
    int n, rows;
    // first pass: coefficients generated in place (amp0 = sqrt(0.023 r0^-5/3) / (n pixel), frequencies
    // in units of the cell 1 / (n pixel), l2 = (n pixel / L0)^2), FFT along kx, complex result
    // stored transposed in dst_c
    float amp0, l2;
    uint32_t key0, key1;
    // second pass: rows of src, FFT along ky, real part stored transposed in dst_r
    const float2* src;
    float2* dst_c;
    float* dst_r;
    const float2* W;
    int radices[16];
    int n_radices;
};

// conj(c_k) of coefficient k = ky n + kx: a_k (z_c - i z_s), a_k = amp0 (kx'^2 + ky'^2 + l2)^(-11/12)
// (the spectrum in cell units), Box-Muller pair of Philox words 0, 1 at counter (k, 0, 0, 1)
__device__ __forceinline__ float2 screen_coeff(int n, int kx, int ky, float amp0, float l2, uint32_t key0,
                                               uint32_t key1) {
    const uint32_t k = (uint32_t)ky * (uint32_t)n + (uint32_t)kx;
    uint32_t w[4] = {k, 0u, 0u, 1u};
    philox4x32_10(w, key0, key1);
    float zc, zs;
    nz_box_muller2(nz_uniform(w[0]), nz_uniform(w[1]), zc, zs);
    const float sx = (float)(kx <= (n - 1) / 2 ? kx : kx - n);
    const float sy = (float)(ky <= (n - 1) / 2 ? ky : ky - n);
    const float a = (kx == 0 && ky == 0) ? 0.0f : amp0 * exp2f(-11.0f / 12.0f * log2f(sx * sx + sy * sy + l2));
    return make_float2(zc * a, -zs * a);
}

// NCT > 0: the transform length is NCT, known at compile time (constant index arithmetic)
template <bool GEN, int NCT>
__global__ void __launch_bounds__(kScreenThreads) screen_fft_pass(ScreenPass P) {
    extern __shared__ float4 smem_raw[];
    const int n = NCT > 0 ? NCT : P.n, rows = NCT > 0 ? screen_rows(NCT) : P.rows;
    float2* A = reinterpret_cast<float2*>(smem_raw);
    float2* B = A + rows * n;
    float2* W = B + rows * n;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int row0 = blockIdx.x * rows;
    for (int q = tid; q < n; q += nthr) W[q] = P.W[q];
    for (int q = tid; q < rows * n; q += nthr) {
        const int r = q / n, c = q - r * n;
        float2 v = make_float2(0.0f, 0.0f);
        if (row0 + r < n) {
            if constexpr (GEN) v = screen_coeff(n, c, row0 + r, P.amp0, P.l2, P.key0, P.key1);
            else v = P.src[(size_t)(row0 + r) * n + c];
        }
        A[q] = v;
    }
    __syncthreads();
    const float2* R;
    if constexpr (NCT > 0) R = fft_tab<NCT>(A, B, rows, W, tid, nthr);
    else R = stockham_fft(A, B, n, P.radices, P.n_radices, rows, n, 1, W, tid, nthr);
    for (int q = tid; q < rows * n; q += nthr) {
        const int c = q / rows, r = q - c * rows;
        if (row0 + r >= n) continue;
        const float2 v = R[r * n + c];
        if constexpr (GEN) P.dst_c[(size_t)c * n + row0 + r] = v;
        else P.dst_r[(size_t)c * n + row0 + r] = v.x;
    }
}

}  // namespace

size_t screen_fft_smem(int n) { return sizeof(float2) * (2 * (size_t)screen_rows(n) * n + n); }

namespace {

template <int NCT>
cudaError_t screen_passes(ScreenPass P, unsigned blocks, cudaStream_t s) {
    const size_t bytes = screen_fft_smem(P.n);
    cudaError_t e = cudaFuncSetAttribute(screen_fft_pass<true, NCT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(screen_fft_pass<false, NCT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    float2* work = P.dst_c;
    float* out = P.dst_r;
    P.dst_r = nullptr;
    screen_fft_pass<true, NCT><<<blocks, kScreenThreads, bytes, s>>>(P);
    P.src = work;
    P.dst_c = nullptr;
    P.dst_r = out;
    screen_fft_pass<false, NCT><<<blocks, kScreenThreads, bytes, s>>>(P);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_screen(int n, double pixel, double r0, double L0, unsigned long long seed, const int* radices,
                          int n_radices, float2* work, float2* W, float* out, cudaStream_t s) {
    // twiddles: stage-major for the compile-time sizes, the plain table otherwise
    switch (n) {
        case 256: screen_stage_twiddles<256><<<1, 256, 0, s>>>(W); break;
        case 512: screen_stage_twiddles<512><<<2, 256, 0, s>>>(W); break;
        case 1024: screen_stage_twiddles<1024><<<4, 256, 0, s>>>(W); break;
        case 2048: screen_stage_twiddles<2048><<<8, 256, 0, s>>>(W); break;
        case 4096: screen_stage_twiddles<4096><<<16, 256, 0, s>>>(W); break;
        default: screen_twiddle_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, W);
    }
    ScreenPass P{};
    P.n = n;
    P.rows = screen_rows(n);
    const double extent = (double)n * pixel;
    P.amp0 = (float)(sqrt(0.023 * pow(r0, -5.0 / 3.0)) * pow(extent, 11.0 / 6.0) / extent);
    P.l2 = (float)((extent / L0) * (extent / L0));
    P.key0 = (uint32_t)seed;
    P.key1 = (uint32_t)(seed >> 32);
    P.W = W;
    P.n_radices = n_radices;
    for (int i = 0; i < n_radices && i < 16; ++i) P.radices[i] = radices[i];
    P.dst_c = work;
    P.dst_r = out;
    const unsigned blocks = (unsigned)((n + P.rows - 1) / P.rows);
    switch (n) {   // the power-of-two sizes get compile-time transforms
        case 256: return screen_passes<256>(P, blocks, s);
        case 512: return screen_passes<512>(P, blocks, s);
        case 1024: return screen_passes<1024>(P, blocks, s);
        case 2048: return screen_passes<2048>(P, blocks, s);
        case 4096: return screen_passes<4096>(P, blocks, s);
        default: return screen_passes<0>(P, blocks, s);
    }
}

}  // namespace mcao
