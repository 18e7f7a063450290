// Test program for the double-single primitives of md_common.cuh (Sec. 2.4,
// Algorithm 1): reads n operand pairs (a.hi, a.lo, b.hi, b.lo as float32) from
// argv[1], evaluates ds_add(a, b), ds_mul(a, b) and ds_mul_f(a, b.hi) on the
// GPU and writes the six result words per pair to argv[2].  Built and run by
// tests/test_ds_arithmetic.py.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "md_common.cuh"

__global__ void k_ds(const float4 *in, float *out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const float4 v = in[i];
    const mdk::ds a = mdk::ds_from(v.x, v.y), b = mdk::ds_from(v.z, v.w);
    const mdk::ds s = mdk::ds_add(a, b), p = mdk::ds_mul(a, b), q = mdk::ds_mul_f(a, v.z);
    out[6 * i + 0] = s.hi; out[6 * i + 1] = s.lo;
    out[6 * i + 2] = p.hi; out[6 * i + 3] = p.lo;
    out[6 * i + 4] = q.hi; out[6 * i + 5] = q.lo;
}

int main(int argc, char **argv)
{
    if (argc != 3)
        return 2;
    FILE *f = fopen(argv[1], "rb");
    if (!f)
        return 3;
    int n = 0;
    if (fread(&n, sizeof n, 1, f) != 1 || n <= 0)
        return 4;
    std::vector<float4> h(n);
    if (fread(h.data(), sizeof(float4), n, f) != (size_t)n)
        return 5;
    fclose(f);
    float4 *din = nullptr;
    float *dout = nullptr;
    if (cudaMalloc(&din, sizeof(float4) * n) != cudaSuccess || cudaMalloc(&dout, sizeof(float) * 6 * n) != cudaSuccess)
        return 6;
    cudaMemcpy(din, h.data(), sizeof(float4) * n, cudaMemcpyHostToDevice);
    k_ds<<<(n + 255) / 256, 256>>>(din, dout, n);
    std::vector<float> o(6 * (size_t)n);
    if (cudaMemcpy(o.data(), dout, sizeof(float) * 6 * n, cudaMemcpyDeviceToHost) != cudaSuccess)
        return 7;
    cudaFree(din);
    cudaFree(dout);
    FILE *g = fopen(argv[2], "wb");
    if (!g || fwrite(o.data(), sizeof(float), o.size(), g) != o.size())
        return 8;
    fclose(g);
    return 0;
}
