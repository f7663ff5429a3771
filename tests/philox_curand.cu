// Test program: Philox4x32-10 outputs of cuRAND's device function for counters and keys given
// on the command line; prints one line of four hex words per input.  Used only by the tests to
// pin the oracle's Philox against an independent implementation.
#include <cstdio>
#include <cstdlib>
#include <curand_kernel.h>

__global__ void run(const uint4* c, const uint2* k, uint4* out, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = curand_Philox4x32_10(c[i], k[i]);
}

int main(int argc, char** argv) {
    int n = (argc - 1) / 6;
    if (n < 1 || n > 1024) return 2;
    uint4* hc = (uint4*)malloc(sizeof(uint4) * n);
    uint2* hk = (uint2*)malloc(sizeof(uint2) * n);
    uint4* ho = (uint4*)malloc(sizeof(uint4) * n);
    for (int i = 0; i < n; ++i) {
        unsigned v[6];
        for (int j = 0; j < 6; ++j) v[j] = (unsigned)strtoul(argv[1 + 6 * i + j], nullptr, 0);
        hc[i] = make_uint4(v[0], v[1], v[2], v[3]);
        hk[i] = make_uint2(v[4], v[5]);
    }
    uint4 *dc, *dout;
    uint2* dk;
    if (cudaMalloc(&dc, sizeof(uint4) * n) || cudaMalloc(&dk, sizeof(uint2) * n) || cudaMalloc(&dout, sizeof(uint4) * n))
        return 3;
    cudaMemcpy(dc, hc, sizeof(uint4) * n, cudaMemcpyHostToDevice);
    cudaMemcpy(dk, hk, sizeof(uint2) * n, cudaMemcpyHostToDevice);
    run<<<(n + 127) / 128, 128>>>(dc, dk, dout, n);
    if (cudaMemcpy(ho, dout, sizeof(uint4) * n, cudaMemcpyDeviceToHost) != cudaSuccess) return 4;
    for (int i = 0; i < n; ++i) printf("%08x %08x %08x %08x\n", ho[i].x, ho[i].y, ho[i].z, ho[i].w);
    return 0;
}
