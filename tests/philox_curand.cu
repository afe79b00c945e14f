// Test helper: CUDA's own Philox4x32-10 (curand_Philox4x32_10 from the
// curand device headers) on counters and keys read from a file, written to
// another: the independent reference that the library's and the oracle's
// Philox are checked against.  Input: n records of 6 u32 (c0 c1 c2 c3 k0 k1),
// output: n records of 4 u32.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include <cuda_runtime.h>
#include <curand_philox4x32_x.h>

__global__ void philox_ref_kernel(const unsigned* in, unsigned* out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned* r = in + 6 * (size_t)i;
    const uint4 v = curand_Philox4x32_10(make_uint4(r[0], r[1], r[2], r[3]),
                                         make_uint2(r[4], r[5]));
    out[4 * (size_t)i] = v.x;
    out[4 * (size_t)i + 1] = v.y;
    out[4 * (size_t)i + 2] = v.z;
    out[4 * (size_t)i + 3] = v.w;
}

int main(int argc, char** argv)
{
    if (argc != 3) return 2;
    FILE* f = std::fopen(argv[1], "rb");
    if (!f) return 3;
    std::vector<unsigned> in;
    unsigned buf[6];
    while (std::fread(buf, sizeof(unsigned), 6, f) == 6) in.insert(in.end(), buf, buf + 6);
    std::fclose(f);
    const int n = (int)(in.size() / 6);
    if (n == 0) return 4;
    unsigned *d_in = nullptr, *d_out = nullptr;
    std::vector<unsigned> out(4 * (size_t)n);
    if (cudaMalloc(&d_in, in.size() * sizeof(unsigned)) != cudaSuccess) return 5;
    if (cudaMalloc(&d_out, out.size() * sizeof(unsigned)) != cudaSuccess) return 5;
    cudaMemcpy(d_in, in.data(), in.size() * sizeof(unsigned), cudaMemcpyHostToDevice);
    philox_ref_kernel<<<(n + 255) / 256, 256>>>(d_in, d_out, n);
    if (cudaMemcpy(out.data(), d_out, out.size() * sizeof(unsigned), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
        return 6;
    cudaFree(d_in);
    cudaFree(d_out);
    FILE* g = std::fopen(argv[2], "wb");
    if (!g) return 7;
    std::fwrite(out.data(), sizeof(unsigned), out.size(), g);
    std::fclose(g);
    return 0;
}
