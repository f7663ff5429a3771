// Tikhonov-regularised least-squares control matrix in FP64 on the GPU ("Control Matrix": the
// reconstructor is a pseudo-inverse of the interaction matrix, and MCAO least squares is
// ill-posed, hence a regularisation coefficient):
//   R = -(D^T D + lambda I)^(-1) D^T,   lambda = alpha tr(D^T D) / n_cmd,
// D [n_slopes][n_cmd] the interaction matrix (float32), R [n_cmd][n_slopes].  The minus sign: D is
// measured with the DM subtracted from the wavefront, and the loop applies c <- c + g R s.
//
// Every step runs in double precision in the kernels below, on 64 x 64 tiles:
//   1. mask of the tiles of D that hold a nonzero (a subaperture sees only the actuators within
//      the influence functions' reach, so most tiles of D are exactly zero);
//   2. Gram matrix G = D^T D, lower tiles, summing only slope tiles where both D tiles are
//      nonzero; mirrored into the upper tiles;
//   3. lambda from the trace, G + lambda I (padding rows past n_cmd get a unit diagonal);
//   4. blocked right-looking Cholesky G = L L^T: per block column k, the diagonal block is
//      factored and inverted in shared memory, the panel below is multiplied by that inverse's
//      transpose, and the trailing lower tiles are updated;
//   5. X = L^(-1) by a right-looking solve of L X = I: per block row i, X[i][j] = Linv_ii X[i][j]
//      for j <= i, then X[m][j] -= L[m][i] X[i][j] below;
//   6. M^(-1) = X^T X (lower tiles, mirrored), written over L;
//   7. R = -M^(-1) D^T, again skipping zero tiles of D; rounded to float32 once, at the store
//      (or stored in double).
// The GB300's FP64 units are slow (about 1.25 TFLOP/s per GPU), so the kernels are plain
// register-blocked tile products (each thread 4 x 4 outputs) bound by the double FMA rate; the
// zero-tile skipping is what keeps the 39 m case (8051 x 55608) to seconds.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>

#include "../../include/mcao.h"

namespace {

constexpr int kT = 64;          // tile side
constexpr int kKC = 32;         // k depth of one shared-memory chunk
constexpr int kThreads = 256;   // 16 x 16 threads, 4 x 4 outputs each

// One chunk of a tile product: As[k][r], Bs[k][c] for k < kKC (rows padded by one double).
struct Chunk {
    double a[kKC][kT + 1];
    double b[kKC][kT + 1];
};

__device__ __forceinline__ void chunk_fma(const Chunk& ch, double (&c)[4][4], int ty, int tx) {
#pragma unroll 8
    for (int k = 0; k < kKC; ++k) {
        double av[4], bv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            av[i] = ch.a[k][ty * 4 + i];
            bv[i] = ch.b[k][tx * 4 + i];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) c[i][j] = fma(av[i], bv[j], c[i][j]);
    }
}

// T[k][i] = src[(r0 + k) ld + c0 + i] for k < kKC, i < 64 (the source block as it is), zero past
// (nr, nc); float or double source
template <typename S>
__device__ __forceinline__ void load_direct(double (*T)[kT + 1], const S* src, long long ld, long long r0, long long c0,
                                            long long nr, long long nc) {
    for (int q = threadIdx.x; q < kKC * kT; q += kThreads) {
        const int k = q / kT, i = q - k * kT;
        const long long r = r0 + k, c = c0 + i;
        T[k][i] = (r < nr && c < nc) ? (double)src[r * ld + c] : 0.0;
    }
}

// T[k][i] = src[(r0 + i) ld + c0 + k] (the source block transposed), zero past (nr, nc)
template <typename S>
__device__ __forceinline__ void load_trans(double (*T)[kT + 1], const S* src, long long ld, long long r0, long long c0,
                                           long long nr, long long nc) {
    for (int q = threadIdx.x; q < kKC * kT; q += kThreads) {
        const int i = q / kKC, k = q - i * kKC;   // consecutive threads walk along a source row
        const long long r = r0 + i, c = c0 + k;
        T[k][i] = (r < nr && c < nc) ? (double)src[r * ld + c] : 0.0;
    }
}

// lower-triangle tile index t -> (i, j), i >= j, i < n
__device__ __forceinline__ void tri_index(long long t, int& i, int& j) {
    int ii = (int)floor((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((long long)(ii + 1) * (ii + 2) / 2 <= t) ++ii;
    while ((long long)ii * (ii + 1) / 2 > t) --ii;
    i = ii;
    j = (int)(t - (long long)ii * (ii + 1) / 2);
}

// 1. mask[S][J] = 1 if the tile (slopes 64 S.., commands 64 J..) of D holds a nonzero
__global__ void __launch_bounds__(kThreads) tik_mask_kernel(const float* __restrict__ D, long long ld, int n_slopes,
                                                            int n_cmd, int nJ, unsigned char* __restrict__ mask) {
    const int J = blockIdx.x, S = blockIdx.y;
    int any = 0;
    for (int q = threadIdx.x; q < kT * kT; q += kThreads) {
        const int r = S * kT + q / kT, c = J * kT + (q % kT);
        if (r < n_slopes && c < n_cmd && D[(long long)r * ld + c] != 0.0f) any = 1;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) mask[(long long)S * nJ + J] = (unsigned char)any;
}

// 2. G[I][J] = sum_s D[s][I..]^T D[s][J..] for lower tiles, mirrored
__global__ void __launch_bounds__(kThreads) tik_gram_kernel(const float* __restrict__ D, long long ld, int n_slopes,
                                                            int n_cmd, int nS, int nt,
                                                            const unsigned char* __restrict__ mask,
                                                            double* __restrict__ G, long long ldg) {
    __shared__ Chunk ch;
    int I, J;
    tri_index(blockIdx.x, I, J);
    const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
    double c[4][4] = {};
    for (int S = 0; S < nS; ++S) {
        if (!mask[(long long)S * nt + I] || !mask[(long long)S * nt + J]) continue;
        for (int k0 = 0; k0 < kT; k0 += kKC) {
            load_direct(ch.a, D, ld, (long long)S * kT + k0, (long long)I * kT, n_slopes, n_cmd);
            load_direct(ch.b, D, ld, (long long)S * kT + k0, (long long)J * kT, n_slopes, n_cmd);
            __syncthreads();
            chunk_fma(ch, c, ty, tx);
            __syncthreads();
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long long r = (long long)I * kT + ty * 4 + i, q = (long long)J * kT + tx * 4 + j;
            G[r * ldg + q] = c[i][j];
            if (I != J) G[q * ldg + r] = c[i][j];
        }
}

// 3. lambda = alpha tr(G) / n_cmd; G + lambda I on the first n_cmd rows, unit diagonal on the
// padding rows (their rows and columns of G are zero)
__global__ void tik_regularize_kernel(double* __restrict__ G, long long ldg, int n_cmd, int npad, double alpha,
                                      double* __restrict__ lambda_out) {
    __shared__ double part[1024];
    double s = 0.0;
    for (int i = threadIdx.x; i < n_cmd; i += blockDim.x) s += G[(long long)i * ldg + i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    const double lam = alpha * part[0] / (double)n_cmd;
    for (int i = threadIdx.x; i < npad; i += blockDim.x) {
        if (i < n_cmd)
            G[(long long)i * ldg + i] += lam;
        else
            G[(long long)i * ldg + i] = 1.0;
    }
    if (threadIdx.x == 0) *lambda_out = lam;
}

// 4a. factor the diagonal block k in shared memory (lower Cholesky), write L_kk over it (upper
// part zero) and its inverse to Linv[k]; a pivot <= 0 sets *err (and is replaced by 1 so the
// remaining steps stay finite)
__global__ void __launch_bounds__(kThreads) tik_potrf_kernel(double* __restrict__ A, long long lda, int k,
                                                             double* __restrict__ Linv, int* __restrict__ err) {
    extern __shared__ double potrf_sm[];
    double(*S)[kT + 1] = reinterpret_cast<double(*)[kT + 1]>(potrf_sm);
    double(*X)[kT + 1] = reinterpret_cast<double(*)[kT + 1]>(potrf_sm + kT * (kT + 1));
    const long long o = (long long)k * kT;
    for (int q = threadIdx.x; q < kT * kT; q += kThreads) S[q / kT][q % kT] = A[(o + q / kT) * lda + o + q % kT];
    __syncthreads();
    for (int j = 0; j < kT; ++j) {
        if (threadIdx.x == 0) {
            double d = S[j][j];
            if (!(d > 0.0)) {
                atomicExch(err, 1);
                d = 1.0;
            }
            S[j][j] = sqrt(d);
        }
        __syncthreads();
        for (int i = j + 1 + threadIdx.x; i < kT; i += kThreads) S[i][j] /= S[j][j];
        __syncthreads();
        // trailing update of the lower part: pairs (i, c), j < c <= i
        const int m = kT - j - 1;
        for (int q = threadIdx.x; q < m * m; q += kThreads) {
            const int i = j + 1 + q / m, c = j + 1 + q % m;
            if (c <= i) S[i][c] -= S[i][j] * S[c][j];
        }
        __syncthreads();
    }
    // inverse of the lower factor: column c solves L x = e_c by forward substitution
    if (threadIdx.x < kT) {
        const int c = threadIdx.x;
        for (int r = 0; r < kT; ++r) {
            double v = (r == c) ? 1.0 : 0.0;
            if (r < c) {
                X[r][c] = 0.0;
                continue;
            }
            for (int q = c; q < r; ++q) v -= S[r][q] * X[q][c];
            X[r][c] = v / S[r][r];
        }
    }
    __syncthreads();
    double* Lk = Linv + (long long)k * kT * kT;
    for (int q = threadIdx.x; q < kT * kT; q += kThreads) {
        const int r = q / kT, c = q % kT;
        A[(o + r) * lda + o + c] = (c <= r) ? S[r][c] : 0.0;
        Lk[q] = X[r][c];
    }
}

// 4b. panel: A[i][k] <- A[i][k] Linv_kk^T for the tiles i > k
__global__ void __launch_bounds__(kThreads) tik_trsm_kernel(double* __restrict__ A, long long lda, int k,
                                                            const double* __restrict__ Linv) {
    __shared__ Chunk ch;
    const int i = k + 1 + blockIdx.x;
    const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
    const long long npad = (long long)kT * (k + 1 + gridDim.x);   // gridDim.x = nt - k - 1
    const double* Lk = Linv + (long long)k * kT * kT;
    double c[4][4] = {};
    for (int k0 = 0; k0 < kT; k0 += kKC) {
        // C[r][q] = sum_m A[i][k][r][m] Linv[q][m]
        load_trans(ch.a, A, lda, (long long)i * kT, (long long)k * kT + k0, npad, npad);
        load_trans(ch.b, Lk, kT, 0, k0, kT, kT);
        __syncthreads();
        chunk_fma(ch, c, ty, tx);
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
            A[((long long)i * kT + ty * 4 + a) * lda + (long long)k * kT + tx * 4 + b] = c[a][b];
}

// 4c. trailing update A[i][j] -= A[i][k] A[j][k]^T for the lower tiles i >= j > k
__global__ void __launch_bounds__(kThreads) tik_update_kernel(double* __restrict__ A, long long lda, int k, int nt) {
    __shared__ Chunk ch;
    int i, j;
    tri_index(blockIdx.x, i, j);
    i += k + 1;
    j += k + 1;
    const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
    const long long npad = (long long)nt * kT;
    double c[4][4] = {};
    for (int k0 = 0; k0 < kT; k0 += kKC) {
        load_trans(ch.a, A, lda, (long long)i * kT, (long long)k * kT + k0, npad, npad);
        load_trans(ch.b, A, lda, (long long)j * kT, (long long)k * kT + k0, npad, npad);
        __syncthreads();
        chunk_fma(ch, c, ty, tx);
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            double* p = &A[((long long)i * kT + ty * 4 + a) * lda + (long long)j * kT + tx * 4 + b];
            *p -= c[a][b];
        }
}

// X = I (the right-hand side of L X = I)
__global__ void tik_eye_kernel(double* __restrict__ X, long long ldx, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        X[i * ldx + i] = 1.0;
}

// 5a. X[i][j] <- Linv_ii X[i][j] for j <= i (in place; all of the block row is read first)
__global__ void __launch_bounds__(kThreads) tik_trinv_scale_kernel(double* __restrict__ X, long long ldx, int i,
                                                                   const double* __restrict__ Linv, int nt) {
    __shared__ Chunk ch;
    const int j = blockIdx.x;
    const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
    const long long npad = (long long)nt * kT;
    const double* Li = Linv + (long long)i * kT * kT;
    double c[4][4] = {};
    for (int k0 = 0; k0 < kT; k0 += kKC) {
        // C[r][q] = sum_m Linv[r][m] X[i][j][m][q]
        load_trans(ch.a, Li, kT, 0, k0, kT, kT);
        load_direct(ch.b, X, ldx, (long long)i * kT + k0, (long long)j * kT, npad, npad);
        __syncthreads();
        chunk_fma(ch, c, ty, tx);
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
            X[((long long)i * kT + ty * 4 + a) * ldx + (long long)j * kT + tx * 4 + b] = c[a][b];
}

// 5b. X[m][j] -= L[m][i] X[i][j] for m > i, j <= i
__global__ void __launch_bounds__(kThreads) tik_trinv_update_kernel(double* __restrict__ X, long long ldx,
                                                                    const double* __restrict__ L, long long ldl, int i,
                                                                    int nt) {
    __shared__ Chunk ch;
    const int m = i + 1 + blockIdx.x / (i + 1), j = blockIdx.x % (i + 1);
    const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
    const long long npad = (long long)nt * kT;
    double c[4][4] = {};
    for (int k0 = 0; k0 < kT; k0 += kKC) {
        load_trans(ch.a, L, ldl, (long long)m * kT, (long long)i * kT + k0, npad, npad);
        load_direct(ch.b, X, ldx, (long long)i * kT + k0, (long long)j * kT, npad, npad);
        __syncthreads();
        chunk_fma(ch, c, ty, tx);
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            double* p = &X[((long long)m * kT + ty * 4 + a) * ldx + (long long)j * kT + tx * 4 + b];
            *p -= c[a][b];
        }
}

// 6. Minv[I][J] = sum_{m >= I} X[m][I]^T X[m][J] for lower tiles (X lower triangular), mirrored
__global__ void __launch_bounds__(kThreads) tik_xtx_kernel(const double* __restrict__ X, long long ldx, int nt,
                                                           double* __restrict__ Minv, long long ldm) {
    __shared__ Chunk ch;
    int I, J;
    tri_index(blockIdx.x, I, J);
    const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
    const long long npad = (long long)nt * kT;
    double c[4][4] = {};
    for (int m = I; m < nt; ++m)
        for (int k0 = 0; k0 < kT; k0 += kKC) {
            load_direct(ch.a, X, ldx, (long long)m * kT + k0, (long long)I * kT, npad, npad);
            load_direct(ch.b, X, ldx, (long long)m * kT + k0, (long long)J * kT, npad, npad);
            __syncthreads();
            chunk_fma(ch, c, ty, tx);
            __syncthreads();
        }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const long long r = (long long)I * kT + ty * 4 + a, q = (long long)J * kT + tx * 4 + b;
            Minv[r * ldm + q] = c[a][b];
            if (I != J) Minv[q * ldm + r] = c[a][b];
        }
}

// 7. R[I..][S..] = -sum_J Minv[I][J] D[S][J]^T over the nonzero tiles of D (Minv symmetric:
// its block (J, I) is read as it is)
template <typename Out>
__global__ void __launch_bounds__(kThreads) tik_apply_kernel(const double* __restrict__ Minv, long long ldm, int nt,
                                                             const float* __restrict__ D, long long ld, int n_slopes,
                                                             int n_cmd, const unsigned char* __restrict__ mask,
                                                             Out* __restrict__ R, long long ldr) {
    __shared__ Chunk ch;
    const int I = blockIdx.x, S = blockIdx.y;
    const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
    const long long npad = (long long)nt * kT;
    double c[4][4] = {};
    for (int J = 0; J < nt; ++J) {
        if (!mask[(long long)S * nt + J]) continue;
        for (int k0 = 0; k0 < kT; k0 += kKC) {
            // C[r][q] = sum_m Minv[J0 + m][I0 + r] D[S0 + q][J0 + m]
            load_direct(ch.a, Minv, ldm, (long long)J * kT + k0, (long long)I * kT, npad, npad);
            load_trans(ch.b, D, ld, (long long)S * kT, (long long)J * kT + k0, n_slopes, n_cmd);
            __syncthreads();
            chunk_fma(ch, c, ty, tx);
            __syncthreads();
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const long long r = (long long)I * kT + ty * 4 + a, q = (long long)S * kT + tx * 4 + b;
            if (r < n_cmd && q < n_slopes) R[r * ldr + q] = (Out)(-c[a][b]);
        }
}

mcao_status report(char* err, size_t err_len, mcao_status st, const char* fmt, ...) {
    if (err && err_len) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(err, err_len, fmt, ap);
        va_end(ap);
    }
    return st;
}

}  // namespace

extern "C" mcao_status mcao_tikhonov_reconstructor(const float* D, int n_slopes, int n_cmd, size_t ld_d, double alpha,
                                                   void* R, size_t ld_r, int r_fp64, void* stream, double* lambda,
                                                   char* err, size_t err_len) {
    if (err && err_len) err[0] = '\0';
    if (!D || !R) return report(err, err_len, MCAO_E_INVALID_ARG, "D and R must be device pointers");
    if (n_slopes < 1 || n_cmd < 1) return report(err, err_len, MCAO_E_SHAPE, "n_slopes and n_cmd must be >= 1");
    if (ld_d < (size_t)n_cmd || ld_r < (size_t)n_slopes)
        return report(err, err_len, MCAO_E_SHAPE, "need ld_d >= n_cmd and ld_r >= n_slopes");
    if (!std::isfinite(alpha) || alpha < 0.0) return report(err, err_len, MCAO_E_INVALID_ARG, "alpha must be >= 0");
    if (r_fp64 != 0 && r_fp64 != 1) return report(err, err_len, MCAO_E_INVALID_ARG, "r_fp64 must be 0 or 1");
    const int nt = (n_cmd + kT - 1) / kT, nS = (n_slopes + kT - 1) / kT;
    const long long npad = (long long)nt * kT;
    cudaStream_t st = (cudaStream_t)stream;
    double *G = nullptr, *X = nullptr, *Linv = nullptr, *d_lam = nullptr;
    unsigned char* mask = nullptr;
    int* d_err = nullptr;
    cudaError_t e = cudaMalloc(&G, sizeof(double) * npad * npad);
    if (e == cudaSuccess) e = cudaMalloc(&X, sizeof(double) * npad * npad);
    if (e == cudaSuccess) e = cudaMalloc(&Linv, sizeof(double) * nt * kT * kT);
    if (e == cudaSuccess) e = cudaMalloc(&mask, (size_t)nS * nt);
    if (e == cudaSuccess) e = cudaMalloc(&d_err, 2 * sizeof(double));   // error flag, then lambda
    auto cleanup = [&]() {
        cudaFree(G);
        cudaFree(X);
        cudaFree(Linv);
        cudaFree(mask);
        cudaFree(d_err);
    };
    if (e != cudaSuccess) {
        cleanup();
        cudaGetLastError();
        return report(err, err_len, e == cudaErrorMemoryAllocation ? MCAO_E_OOM : MCAO_E_CUDA,
                      "allocation of the FP64 work arrays (%lld x %lld doubles, twice): %s", npad, npad,
                      cudaGetErrorString(e));
    }
    d_lam = reinterpret_cast<double*>(d_err) + 1;
    const int potrf_smem = 2 * kT * (kT + 1) * (int)sizeof(double);
    e = cudaFuncSetAttribute(tik_potrf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, potrf_smem);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(G, 0, sizeof(double) * npad * npad, st);
    if (e == cudaSuccess) {
        tik_mask_kernel<<<dim3(nt, nS), kThreads, 0, st>>>(D, (long long)ld_d, n_slopes, n_cmd, nt, mask);
        tik_gram_kernel<<<(unsigned)((long long)nt * (nt + 1) / 2), kThreads, 0, st>>>(
            D, (long long)ld_d, n_slopes, n_cmd, nS, nt, mask, G, npad);
        tik_regularize_kernel<<<1, 1024, 0, st>>>(G, npad, n_cmd, (int)npad, alpha, d_lam);
        for (int k = 0; k < nt; ++k) {
            tik_potrf_kernel<<<1, kThreads, potrf_smem, st>>>(G, npad, k, Linv, d_err);
            const int rest = nt - k - 1;
            if (rest > 0) {
                tik_trsm_kernel<<<rest, kThreads, 0, st>>>(G, npad, k, Linv);
                tik_update_kernel<<<(unsigned)((long long)rest * (rest + 1) / 2), kThreads, 0, st>>>(G, npad, k, nt);
            }
        }
        e = cudaGetLastError();
    }
    // X = L^-1: start from the identity
    if (e == cudaSuccess) e = cudaMemsetAsync(X, 0, sizeof(double) * npad * npad, st);
    if (e == cudaSuccess) {
        tik_eye_kernel<<<64, 256, 0, st>>>(X, npad, npad);
        for (int i = 0; i < nt; ++i) {
            tik_trinv_scale_kernel<<<i + 1, kThreads, 0, st>>>(X, npad, i, Linv, nt);
            const int below = nt - i - 1;
            if (below > 0) tik_trinv_update_kernel<<<below * (i + 1), kThreads, 0, st>>>(X, npad, G, npad, i, nt);
        }
        // M^-1 over the factor
        tik_xtx_kernel<<<(unsigned)((long long)nt * (nt + 1) / 2), kThreads, 0, st>>>(X, npad, nt, G, npad);
        if (r_fp64)
            tik_apply_kernel<double><<<dim3(nt, nS), kThreads, 0, st>>>(G, npad, nt, D, (long long)ld_d, n_slopes,
                                                                        n_cmd, mask, (double*)R, (long long)ld_r);
        else
            tik_apply_kernel<float><<<dim3(nt, nS), kThreads, 0, st>>>(G, npad, nt, D, (long long)ld_d, n_slopes,
                                                                       n_cmd, mask, (float*)R, (long long)ld_r);
        e = cudaGetLastError();
    }
    int h_err = 0;
    double h_lam = 0.0;
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemcpy(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&h_lam, d_lam, sizeof(double), cudaMemcpyDeviceToHost);
    cleanup();
    if (e != cudaSuccess) return report(err, err_len, MCAO_E_CUDA, "Tikhonov reconstructor: %s", cudaGetErrorString(e));
    if (lambda) *lambda = h_lam;
    if (h_err)
        return report(err, err_len, MCAO_E_UNSUPPORTED,
                      "D^T D + lambda I is not positive definite in double precision (lambda = %g): raise alpha", h_lam);
    return MCAO_OK;
}
