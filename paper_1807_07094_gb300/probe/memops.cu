// memops.cu -- throughput ceilings of the tracer's per-segment memory pattern
// on this GPU (a measurement aid for the roofline discussion, not part of
// libarc).  Every op touches one 32-byte cell record in a 512 MB array
// (larger than L2): modes
//   0  16-byte load of the record's first half
//   1  16-byte vector atomic add with return on its second half
//   2  load of the first half, then the atomic on the second half (the
//      tracer's segment: optical depth read, absorbed photons added)
// Record indices are hashed per lane and walk runs of `run` consecutive
// records (run 1: fully random; longer runs: the locality of a ray crossing
// neighbouring cells).  All indices are reduced modulo the record count.
// Prints one JSON line per (mode, run) with operations per second.
#include <cstdio>
#include <cuda_runtime.h>

__device__ __forceinline__ unsigned mix32(unsigned x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}
__device__ __forceinline__ float4 atom_v4(float4* a, float4 v) {
    float4 o;
    asm volatile("atom.global.add.v4.f32 {%0,%1,%2,%3}, [%4], {%5,%6,%7,%8};"
                 : "=f"(o.x), "=f"(o.y), "=f"(o.z), "=f"(o.w)
                 : "l"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w));
    return o;
}

template <int MODE>
__global__ void k_ops(float4* rec, unsigned nrec, int iters, int run, float* sink) {
    const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned base = mix32(tid * 2654435761u + 12345u);
    float acc = 0.f;
    for (int i = 0; i < iters; ++i) {
        const unsigned r = (mix32(base + (unsigned)(i / run)) + (unsigned)(i % run)) % nrec;
        float4* p = rec + 2 * (size_t)r;
        if (MODE == 0) {
            acc += __ldg(p).x;
        } else if (MODE == 1) {
            acc += atom_v4(p + 1, make_float4(1.f, 1.f, 1.f, 0.f)).x;
        } else {
            const float4 k = __ldg(p);
            acc += atom_v4(p + 1, make_float4(k.x + 1.f, 1.f, 1.f, 0.f)).x;
        }
    }
    if (acc == 1234.5f) sink[0] = acc;   // keeps the loop alive
}

int main() {
    const unsigned nrec = 1u << 24;   // 16M records x 32 B = 512 MB
    float4* rec = nullptr;
    float* sink = nullptr;
    if (cudaMalloc(&rec, (size_t)nrec * 32) != cudaSuccess || cudaMalloc(&sink, 4) != cudaSuccess) return 1;
    cudaMemset(rec, 0, (size_t)nrec * 32);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const char* names[3] = {"load16", "atom16", "load16+atom16"};
    const int threads = 256, blocks = sms * 4, iters = 256, reps = 5;
    for (int run : {1, 8, 32}) {
        for (int mode = 0; mode < 3; ++mode) {
            auto launch = [&]() {
                if (mode == 0) k_ops<0><<<blocks, threads>>>(rec, nrec, iters, run, sink);
                if (mode == 1) k_ops<1><<<blocks, threads>>>(rec, nrec, iters, run, sink);
                if (mode == 2) k_ops<2><<<blocks, threads>>>(rec, nrec, iters, run, sink);
            };
            launch();   // warm-up
            cudaEventRecord(e0);
            for (int r = 0; r < reps; ++r) launch();
            cudaEventRecord(e1);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double ops = (double)reps * blocks * threads * iters;
            printf("{\"mode\": \"%s\", \"run\": %d, \"gops\": %.3f}\n", names[mode], run, ops / (ms * 1e6));
        }
    }
    const cudaError_t err = cudaDeviceSynchronize();
    cudaFree(rec);
    cudaFree(sink);
    return err == cudaSuccess ? 0 : 1;
}
