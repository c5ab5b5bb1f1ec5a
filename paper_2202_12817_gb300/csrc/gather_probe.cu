// Random-gather ceilings of this GPU's L2 -> SM path, the bound that the harmonic-sum gathers
// meet before HBM bandwidth: each order of the greedy form reads, per fundamental, bins that lie
// in their own 32-byte sector.  A standalone measurement program (built next to libhs.so, run by
// bench.py): it reads a 32 MB L2-resident buffer with 2048 threads per SM and prints one JSON
// object with the sustained lane-load rate of each access pattern.
//   rand4      every lane a random 4-byte load
//   rand16     every lane a random aligned 16-byte load
//   pair_line  lanes 2i, 2i+1 read two sectors of one random 128-byte line
//   quad_line  lanes 4i..4i+3 read the four sectors of one random line
//   chain      a dependent chain (the next address depends on the loaded value)
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

namespace {

__device__ __forceinline__ uint32_t mix32(uint32_t a)
{
    a ^= a >> 16;
    a *= 0x7feb352dU;
    a ^= a >> 15;
    a *= 0x846ca68bU;
    a ^= a >> 16;
    return a;
}

template <int MODE>
__global__ void k_probe(const float *__restrict__ x, uint32_t mask, int iters, float *out)
{
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31;
    float acc = 0.f;
    uint32_t idx = mix32(tid * 2654435761u) & mask;
    for (int k = 0; k < iters; k += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t key = tid * 64 + k + u;
            if (MODE == 0) {
                acc += __ldg(x + (mix32(key) & mask));
            } else if (MODE == 1) {
                const float4 v = __ldg(reinterpret_cast<const float4 *>(x) + ((mix32(key) & mask) >> 2));
                acc += v.x + v.w;
            } else if (MODE == 2) {
                const uint32_t line = (mix32((tid >> 1) * 64 + k + u) & mask) & ~31u;
                acc += __ldg(x + line + (lane & 1) * 8);
            } else if (MODE == 3) {
                const uint32_t line = (mix32((tid >> 2) * 64 + k + u) & mask) & ~31u;
                acc += __ldg(x + line + (lane & 3) * 8);
            } else {
                const float v = __ldg(x + idx);
                idx = mix32(idx + __float_as_uint(v)) & mask;
                acc += v;
            }
        }
    }
    if (acc == 1234.5f) out[tid] = acc;   // keeps the loads; never true for the zero buffer
}

template <int MODE>
float time_mode(const float *x, uint32_t mask, int blocks, int threads, int iters, float *out)
{
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    for (int w = 0; w < 2; ++w) k_probe<MODE><<<blocks, threads>>>(x, mask, iters, out);
    cudaEventRecord(a);
    k_probe<MODE><<<blocks, threads>>>(x, mask, iters, out);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms;
}

}  // namespace

int main()
{
    const uint32_t n = 1u << 23;   // 32 MB of floats: resident in L2 after the warm-up launches
    const int threads = 256, per_sm = 2048, iters = 64;
    int sms = 0;
    float *x = nullptr, *out = nullptr;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess || sms < 1) {
        std::printf("{\"error\": \"no device\"}\n");
        return 1;
    }
    const int blocks = sms * per_sm / threads;
    const size_t lanes = static_cast<size_t>(blocks) * threads;
    if (cudaMalloc(&x, n * sizeof(float)) != cudaSuccess || cudaMalloc(&out, lanes * sizeof(float)) != cudaSuccess ||
        cudaMemset(x, 0, n * sizeof(float)) != cudaSuccess) {
        std::printf("{\"error\": \"allocation\"}\n");
        return 1;
    }
    const uint32_t mask = n - 1;
    const double loads = static_cast<double>(lanes) * iters;
    const float m0 = time_mode<0>(x, mask, blocks, threads, iters, out);
    const float m1 = time_mode<1>(x, mask, blocks, threads, iters, out);
    const float m2 = time_mode<2>(x, mask, blocks, threads, iters, out);
    const float m3 = time_mode<3>(x, mask, blocks, threads, iters, out);
    const float m4 = time_mode<4>(x, mask, blocks, threads, iters, out);
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        std::printf("{\"error\": \"%s\"}\n", cudaGetErrorString(e));
        return 1;
    }
    // lane-loads per second; pair_line and quad_line carry 2 and 4 sectors per 128-byte line
    std::printf("{\"sms\": %d, \"threads_per_sm\": %d, \"rand4\": %.4e, \"rand16\": %.4e, \"pair_line\": %.4e, "
                "\"quad_line\": %.4e, \"chain\": %.4e, \"chain_latency_ns\": %.1f, "
                "\"line_requests_per_s\": %.4e, \"sectors_per_s\": %.4e}\n",
                sms, per_sm, loads / (m0 * 1e-3), loads / (m1 * 1e-3), loads / (m2 * 1e-3), loads / (m3 * 1e-3),
                loads / (m4 * 1e-3), m4 * 1e6 / iters,
                // the line-request ceiling: random lines with one sector each (max of the single- and
                // two-sector patterns); the sector ceiling: four sectors per line
                (loads / (m0 * 1e-3) > loads / (m2 * 1e-3) / 2 ? loads / (m0 * 1e-3) : loads / (m2 * 1e-3) / 2),
                loads / (m3 * 1e-3));
    cudaFree(x);
    cudaFree(out);
    return 0;
}
