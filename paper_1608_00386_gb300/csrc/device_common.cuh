// Device helpers shared by the wavefront-sensor and science kernels: cone-beam sampling of
// layers and DM surfaces, in-shared-memory Stockham FFT stages, and the detector-noise sampler.
#pragma once

#include <stdint.h>

#include "mcao_internal.h"

namespace mcao {

// ---------------------------------------------------------------------------------------------
// Geometric propagation ("The open loop wave-front measurements" of arXiv:1608.00386: geometric
// projection of each layer, laser guide star at finite distance).  A pupil point x seen along
// direction theta from a source at height H crosses altitude h at x (1 - h/H) + h theta
// (H infinite for natural stars); layers move by (k dt) v.  The host turns that map into Q32.32
// fixed-point grid coordinates (GridView); the kernels evaluate, for a T x T tile of pupil
// samples, one axis entry per grid and per tile column / row (bilinear sampling is separable in
// x and y), then every sample of the tile reads its two entries per grid.
// ---------------------------------------------------------------------------------------------
struct AxisEnt {
    int idx;     // i0 | (i1 << 16): the two neighbouring grid indices
    float t;     // weight of i1
};

__device__ __forceinline__ AxisEnt axis_entry(long long X, int n, int periodic, float inv_n) {
    int i = (int)(X >> 32);
    float t = __uint2float_rn((unsigned)(X & 0xffffffffull)) * 2.3283064365386963e-10f;  // 2^-32
    int i1;
    if (periodic) {
        // i mod n: quotient from the float reciprocal (off by at most a few for |i| < 2^31),
        // then exact integer corrections
        const int q = __float2int_rd(__int2float_rn(i) * inv_n);
        i -= q * n;
        while (i < 0) i += n;
        while (i >= n) i -= n;
        i1 = (i + 1 == n) ? 0 : i + 1;
    } else {
        if (i < 0) {
            i = 0;
            t = 0.0f;
        } else if (i >= n - 1) {
            i = n - 2;
            t = 1.0f;
        }
        i1 = i + 1;
    }
    AxisEnt e;
    e.idx = i | (i1 << 16);
    e.t = t;
    return e;
}

// entries of every grid for the T x T tile with origin (i0, j0): ex[g T + x], ey[g T + y]
template <int T>
__device__ __forceinline__ void tile_entries(const GridView* V, int n_grids, long long k, int i0, int j0,
                                             AxisEnt* ex, AxisEnt* ey, int tid, int nthr) {
    for (int e = tid; e < n_grids * 2 * T; e += nthr) {
        const int g = e / (2 * T), r = e - g * 2 * T;
        const GridView& v = V[g];
        if (r < T) {
            ex[g * T + r] = axis_entry(v.ax + (long long)(i0 + r) * v.bp + k * v.vx, v.n, v.periodic, v.inv_n);
        } else {
            const int y = r - T;
            ey[g * T + y] = axis_entry(v.ay + (long long)(j0 + y) * v.bp + k * v.vy, v.n, v.periodic, v.inv_n);
        }
    }
}

__device__ __forceinline__ float bilinear(const float* data, int n, AxisEnt ex, AxisEnt ey) {
    const int x0 = ex.idx & 0xffff, x1 = ex.idx >> 16;
    const float* r0 = data + (ey.idx & 0xffff) * n;
    const float* r1 = data + (ey.idx >> 16) * n;
    float a = __ldg(r0 + x0), b = __ldg(r0 + x1), c = __ldg(r1 + x0), d = __ldg(r1 + x1);
    float top = fmaf(ex.t, b - a, a);
    float bot = fmaf(ex.t, d - c, c);
    return fmaf(ey.t, bot - top, top);
}

// residual phase (layers - DMs) at tile sample (x, y)
__device__ __forceinline__ float tile_phase(const GridView* V, int n_grids, const AxisEnt* ex,
                                            const AxisEnt* ey, int T, int x, int y) {
    float phi = 0.0f;
#pragma unroll 4
    for (int g = 0; g < n_grids; ++g) {
        float v = bilinear(V[g].data, V[g].n, ex[g * T + x], ey[g * T + y]);
        phi = fmaf(V[g].sign, v, phi);
    }
    return phi;
}

// ---------------------------------------------------------------------------------------------
// Stockham autosort FFT stage in shared memory (forward, exp(-2 pi i ...)), batched.
// Stage with radix R and current sub-transform length ns: for j < N/R, inputs
// src[j + r N/R], twiddle exp(-2 pi i r (j mod ns) / (ns R)), R-point DFT, outputs to
// dst[(j/ns) ns R + (j mod ns) + r ns].  W holds exp(-2 pi i m / N), m < N.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

template <int R>
__device__ __forceinline__ void small_dft(float2* v);

template <>
__device__ __forceinline__ void small_dft<2>(float2* v) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

template <>
__device__ __forceinline__ void small_dft<4>(float2* v) {
    float2 a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
    float2 a2 = cadd(v[1], v[3]), d = csub(v[1], v[3]);
    float2 a3 = make_float2(d.y, -d.x);  // -i (v1 - v3)
    v[0] = cadd(a0, a2);
    v[2] = csub(a0, a2);
    v[1] = cadd(a1, a3);
    v[3] = csub(a1, a3);
}

template <>
__device__ __forceinline__ void small_dft<3>(float2* v) {
    const float c = -0.5f, s = -0.866025403784438647f;  // exp(-2 pi i / 3)
    float2 a = v[0], b = v[1], d = v[2];
    float2 sum = cadd(b, d), dif = csub(b, d);
    v[0] = cadd(a, sum);
    float2 m = make_float2(a.x + c * sum.x, a.y + c * sum.y);
    float2 rot = make_float2(-s * dif.y, s * dif.x);  // i s (b - d)
    v[1] = cadd(m, rot);
    v[2] = csub(m, rot);
}

template <>
__device__ __forceinline__ void small_dft<5>(float2* v) {
    // exp(-2 pi i q / 5), q = 0..4
    const float cr[5] = {1.0f, 0.309016994374947424f, -0.809016994374947424f, -0.809016994374947424f,
                         0.309016994374947424f};
    const float ci[5] = {0.0f, -0.951056516295153572f, -0.587785252292473129f, 0.587785252292473129f,
                         0.951056516295153572f};
    float2 in[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) in[q] = v[q];
#pragma unroll
    for (int r = 0; r < 5; ++r) {
        float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            int m = (q * r) % 5;
            acc.x += in[q].x * cr[m] - in[q].y * ci[m];
            acc.y += in[q].x * ci[m] + in[q].y * cr[m];
        }
        v[r] = acc;
    }
}

// One stage for `batch` transforms of length N; transform f starts at f * fstride and its
// element e sits at e * estride (both in float2 units).
template <int R>
__device__ __forceinline__ void stockham_stage(const float2* src, float2* dst, int N, int ns, int batch,
                                               int fstride, int estride, const float2* W, int tid,
                                               int nthr) {
    const int NR = N / R;
    const int twstep = N / (ns * R);
    for (int idx = tid; idx < batch * NR; idx += nthr) {
        int f = idx / NR, j = idx - f * NR;
        const float2* s = src + (long long)f * fstride;
        float2* d = dst + (long long)f * fstride;
        int k = j % ns;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = s[(j + r * NR) * estride];
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmul(v[r], W[(r * k * twstep) % N]);
        small_dft<R>(v);
        int base = (j / ns) * ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) d[(base + r * ns) * estride] = v[r];
    }
}

// Full transform through the radix list; returns the buffer holding the result (a or b).
// Every stage is followed by a block-wide barrier.
__device__ __forceinline__ float2* stockham_fft(float2* a, float2* b, int N, const int* radices,
                                                int n_radices, int batch, int fstride, int estride,
                                                const float2* W, int tid, int nthr) {
    int ns = 1;
    float2* src = a;
    float2* dst = b;
    for (int q = 0; q < n_radices; ++q) {
        int R = radices[q];
        if (R == 4) stockham_stage<4>(src, dst, N, ns, batch, fstride, estride, W, tid, nthr);
        else if (R == 2) stockham_stage<2>(src, dst, N, ns, batch, fstride, estride, W, tid, nthr);
        else if (R == 5) stockham_stage<5>(src, dst, N, ns, batch, fstride, estride, W, tid, nthr);
        else stockham_stage<3>(src, dst, N, ns, batch, fstride, estride, W, tid, nthr);
        __syncthreads();
        ns *= R;
        float2* t = src;
        src = dst;
        dst = t;
    }
    return src;
}

// Compile-time Stockham: the same stages with N, the sub-transform length and the radix known
// at compile time (index arithmetic by constants, no twiddle modulo).  Radices are taken as
// 4 while possible, then 2, 5, 3, matching the host's factorisation.
__host__ __device__ constexpr int ct_radix(int m) {
    return (m % 4 == 0) ? 4 : (m % 2 == 0) ? 2 : (m % 5 == 0) ? 5 : 3;
}

template <int N, int NS, int R>
__device__ __forceinline__ void stockham_stage_ct(const float2* src, float2* dst, int batch, int fstride,
                                                  const float2* W, int tid, int nthr) {
    constexpr int NR = N / R;
    constexpr int TW = N / (NS * R);
    for (int idx = tid; idx < batch * NR; idx += nthr) {
        const int f = idx / NR, j = idx - f * NR;
        const float2* s = src + (long long)f * fstride;
        float2* d = dst + (long long)f * fstride;
        const int k = j % NS;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = s[j + r * NR];
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmul(v[r], W[r * k * TW]);
        small_dft<R>(v);
        const int base = (j / NS) * NS * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) d[base + r * NS] = v[r];
    }
}

// returns the buffer holding the result; a block-wide barrier follows every stage
template <int N, int NS = 1>
__device__ __forceinline__ float2* stockham_fft_ct(float2* a, float2* b, int batch, int fstride, const float2* W,
                                                   int tid, int nthr) {
    if constexpr (NS >= N) {
        return a;
    } else {
        constexpr int R = ct_radix(N / NS);
        stockham_stage_ct<N, NS, R>(a, b, batch, fstride, W, tid, nthr);
        __syncthreads();
        return stockham_fft_ct<N, NS * R>(b, a, batch, fstride, W, tid, nthr);
    }
}

// The compile-time transform again, with its twiddles in a stage-major table so that a warp's
// butterflies (consecutive k) read consecutive entries instead of one bank at stride N/(ns R):
// for the stage of sub-length ns and radix R, entry off + (r - 1) ns + k holds
// exp(-2 pi i r k / (ns R)) = W[r k N / (ns R)], r = 1 .. R-1, k < ns; off is the sum of the
// earlier stages' ns (R - 1); N - 1 entries in all (stage_twiddle_count).
__host__ __device__ constexpr int stage_twiddle_count(int N) {
    int c = 0;
    for (int ns = 1; ns < N; ns *= ct_radix(N / ns)) c += ns * (ct_radix(N / ns) - 1);
    return c;
}

template <int N, int NS, int R>
__device__ __forceinline__ void stage_tab(const float2* src, float2* dst, int batch, const float2* T, int tid,
                                          int nthr) {
    constexpr int NR = N / R;
    for (int idx = tid; idx < batch * NR; idx += nthr) {
        const int f = idx / NR, j = idx - f * NR;
        const float2* sp = src + f * N;
        float2* dp = dst + f * N;
        const int k = j % NS;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = sp[j + r * NR];
        if constexpr (NS > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], T[(r - 1) * NS + k]);
        }
        small_dft<R>(v);
        const int base = (j / NS) * NS * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dp[base + r * NS] = v[r];
    }
}

// the compile-time Stockham transform reading the stage-major table; returns the buffer holding
// the result (a block-wide barrier follows every stage)
template <int N, int NS = 1, int OFF = 0>
__device__ __forceinline__ float2* fft_tab(float2* a, float2* b, int batch, const float2* T, int tid, int nthr) {
    if constexpr (NS >= N) {
        return a;
    } else {
        constexpr int R = ct_radix(N / NS);
        stage_tab<N, NS, R>(a, b, batch, T + OFF, tid, nthr);
        __syncthreads();
        return fft_tab<N, NS * R, OFF + NS * (R - 1)>(b, a, batch, T, tid, nthr);
    }
}

// ---------------------------------------------------------------------------------------------
// Detector noise.  Counter-based Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) keyed by the
// seed; float sampler with a fixed operation order written with round-to-nearest intrinsics
// (never contracted), so one float intensity maps to one integer.  Pixels go in pairs (o and
// o + n_det^2 / 2 of a subaperture frame, counter word 0 = frame index of o):
//   draw A (counter word 3 = 0): words 0, 1 the two inversion uniforms; words 2, 3 one
//     Box-Muller pair, the two pixels' read noise rint(sigma z), formed when read noise is on;
//   draw B (counter word 3 = 2, only when a pixel has lambda >= 16): words 2, 3 one Box-Muller
//     pair, the photon normals;
//   lambda < 16: Poisson by inversion, p0 = exp(-lambda), p_{k+1} = p_k fl(lambda fl(1/(k+1))),
//                smallest k with u <= F_k (k <= 64);
//   lambda >= 16: max(0, rint(lambda + sqrt(lambda) y)).
// exp: Cody-Waite reduction by ln 2 (two-part constant) and a degree-7 Taylor polynomial; log:
// mantissa in [sqrt(1/2), sqrt(2)) and the atanh series to s^9, s = (m - 1) fl(1/(m + 1));
// cos and sin of 2 pi u: quadrant reduction and Taylor polynomials of sin / cos on [-pi/4, pi/4].
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        unsigned long long p0 = 0xD2511F53ull * (unsigned long long)c[0];
        unsigned long long p1 = 0xCD9E8D57ull * (unsigned long long)c[2];
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0, n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = (uint32_t)p1;
        c[2] = n2;
        c[3] = (uint32_t)p0;
        if (r < 9) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
    }
}

__device__ __forceinline__ float nz_uniform(uint32_t w) {
    return __fmul_rn(__fadd_rn(__uint2float_rn(w >> 8), 0.5f), 5.9604644775390625e-8f);
}

__device__ __forceinline__ float nz_exp(float x) {
    float kf = rintf(__fmul_rn(x, 1.44269502f));
    float r = __fmaf_rn(-kf, 0.693145752f, x);
    r = __fmaf_rn(-kf, 1.42860677e-06f, r);
    float p = 1.98412701e-04f;            // 1/5040
    p = __fmaf_rn(p, r, 1.38888892e-03f); // 1/720
    p = __fmaf_rn(p, r, 8.33333377e-03f); // 1/120
    p = __fmaf_rn(p, r, 4.16666679e-02f); // 1/24
    p = __fmaf_rn(p, r, 1.66666672e-01f); // 1/6
    p = __fmaf_rn(p, r, 0.5f);
    p = __fmaf_rn(p, r, 1.0f);
    p = __fmaf_rn(p, r, 1.0f);
    int k = (int)kf;
    if (k < -126) return 0.0f;
    return __fmul_rn(p, __uint_as_float((uint32_t)(k + 127) << 23));
}

__device__ __forceinline__ float nz_log(float u) {
    uint32_t b = __float_as_uint(u);
    int e = (int)((b >> 23) & 0xffu) - 127;
    float m = __uint_as_float((b & 0x007fffffu) | 0x3f800000u);
    if (m > 1.41421356f) {
        m = __fmul_rn(m, 0.5f);
        e += 1;
    }
    float s = __fmul_rn(__fsub_rn(m, 1.0f), __frcp_rn(__fadd_rn(m, 1.0f)));
    float s2 = __fmul_rn(s, s);
    float p = 1.11111112e-01f;              // 1/9
    p = __fmaf_rn(p, s2, 1.42857149e-01f);  // 1/7
    p = __fmaf_rn(p, s2, 2.00000003e-01f);  // 1/5
    p = __fmaf_rn(p, s2, 3.33333343e-01f);  // 1/3
    p = __fmaf_rn(p, s2, 1.0f);
    float lm = __fmul_rn(__fmul_rn(2.0f, s), p);
    float ef = (float)e;
    return __fmaf_rn(ef, 0.693145752f, __fmaf_rn(ef, 1.42860677e-06f, lm));
}

__device__ __forceinline__ float nz_sin_poly(float y) {
    float y2 = __fmul_rn(y, y);
    float p = 2.75573188e-06f;               // 1/362880
    p = __fmaf_rn(p, y2, -1.98412701e-04f);  // -1/5040
    p = __fmaf_rn(p, y2, 8.33333377e-03f);   // 1/120
    p = __fmaf_rn(p, y2, -1.66666672e-01f);  // -1/6
    return __fmaf_rn(__fmul_rn(p, y2), y, y);
}

__device__ __forceinline__ float nz_cos_poly(float y) {
    float y2 = __fmul_rn(y, y);
    float p = 2.48015876e-05f;               // 1/40320
    p = __fmaf_rn(p, y2, -1.38888892e-03f);  // -1/720
    p = __fmaf_rn(p, y2, 4.16666679e-02f);   // 1/24
    p = __fmaf_rn(p, y2, -0.5f);
    return __fmaf_rn(p, y2, 1.0f);
}

// (cos 2 pi u, sin 2 pi u) for u in [0, 1]: quadrant q = rint(4u), y = 2 pi (u - q/4) (exact
// subtraction), both polynomials, then the quadrant's signs and swap
__device__ __forceinline__ void nz_sincos2pi(float u, float& c, float& s) {
    const float twopi = 6.28318548f;
    const float qf = rintf(__fmul_rn(4.0f, u));
    const float y = __fmul_rn(__fsub_rn(u, __fmul_rn(0.25f, qf)), twopi);
    const float sp = nz_sin_poly(y), cp = nz_cos_poly(y);
    const int q = ((int)qf) & 3;
    const float a = (q & 1) ? sp : cp, b = (q & 1) ? cp : sp;   // cos, sin of y + (q & 1) pi / 2 up to sign
    c = (q == 1 || q == 2) ? -a : a;
    s = (q >= 2) ? -b : b;
}

// two independent standard normals: r = sqrt(-2 log u0), (r cos 2 pi u1, r sin 2 pi u1)
__device__ __forceinline__ void nz_box_muller2(float u0, float u1, float& zc, float& zs) {
    const float rad = __fsqrt_rn(__fmul_rn(-2.0f, nz_log(u0)));
    float c, s;
    nz_sincos2pi(u1, c, s);
    zc = __fmul_rn(rad, c);
    zs = __fmul_rn(rad, s);
}

// recip[j] = fl(1/j), j = 0..65 (entry 0 unused), filled with correctly rounded divisions
constexpr int kRecipEntries = 66;
__device__ __forceinline__ void fill_recip(float* recip, int tid, int nthr) {
    for (int j = tid; j < kRecipEntries; j += nthr) recip[j] = (j > 0) ? __fdiv_rn(1.0f, (float)j) : 0.0f;
}

// Photon count of one pixel: Poisson by inversion for lambda < 16 (uniform u; two terms per
// pass, formed in the same order as one at a time, stopping at the same k), else
// max(0, rint(lambda + sqrt(lambda) y)) with the standard normal y.
__device__ __forceinline__ int nz_photons(float lam, float u, float y, const float* recip) {
    if (lam < 16.0f) {
        float p = nz_exp(-lam), F = p;
        int k = 0;
        while (F < u && k < 64) {
            const float qa = __fmul_rn(lam, recip[k + 1]), qb = __fmul_rn(lam, recip[k + 2]);
            const float pa = __fmul_rn(p, qa), Fa = __fadd_rn(F, pa);
            if (!(Fa < u) || k + 1 >= 64) {
                k += 1;
                break;
            }
            p = __fmul_rn(pa, qb);
            F = __fadd_rn(Fa, p);
            k += 2;
        }
        return k;
    }
    const int n = __float2int_rn(__fmaf_rn(__fsqrt_rn(lam), y, lam));
    return n < 0 ? 0 : n;
}

// Noisy counts of a pixel pair (pixel o and o + n_det^2 / 2 of one subaperture frame; g the
// frame index of pixel o): draw A = Philox(g, step, sensor, 0) gives the two inversion uniforms
// (words 0, 1) and, when read noise is on, one Box-Muller pair (words 2, 3) whose outputs are
// the two pixels' read noise; draw B = Philox(g, step, sensor, 2), formed only when a pixel has
// lambda >= 16, gives one Box-Muller pair (words 2, 3) for the two photon normals.
__device__ __forceinline__ void noise_pair(float lam_a, float lam_b, float read_noise, uint32_t g, uint32_t step,
                                           uint32_t sensor, unsigned long long seed, const float* recip, int& na,
                                           int& nb) {
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    uint32_t w[4] = {g, step, sensor, 0u};
    philox4x32_10(w, k0, k1);
    float ya = 0.0f, yb = 0.0f;
    if (!(lam_a < 16.0f) || !(lam_b < 16.0f)) {
        uint32_t v[4] = {g, step, sensor, 2u};
        philox4x32_10(v, k0, k1);
        nz_box_muller2(nz_uniform(v[2]), nz_uniform(v[3]), ya, yb);
    }
    na = nz_photons(lam_a, nz_uniform(w[0]), ya, recip);
    nb = nz_photons(lam_b, nz_uniform(w[1]), yb, recip);
    if (read_noise > 0.0f) {
        float za, zb;
        nz_box_muller2(nz_uniform(w[2]), nz_uniform(w[3]), za, zb);
        na += __float2int_rn(__fmul_rn(read_noise, za));
        nb += __float2int_rn(__fmul_rn(read_noise, zb));
    }
}

// warp sum
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace mcao
