// Gather roofline probe: the memory access pattern of the walk without its
// arithmetic.  Every thread follows two chains of dependent random reads of
// 64-byte records (two 256-bit loads each, as the walk reads a row record)
// or of 32-byte records (one 256-bit load, the compact table's records);
// the next record index comes from the record just read.  Records per second
// at a given footprint and occupancy bound what the walk kernel can reach.
#include <cstring>

#include "kernels.h"
#include "mcmi.h"

namespace mcmi {

namespace {

__device__ __forceinline__ uint32_t mix32(uint32_t x)
{
    x ^= x >> 16; x *= 0x7FEB352Du;
    x ^= x >> 15; x *= 0x846CA68Bu;
    x ^= x >> 16;
    return x;
}

// n16: 16-byte words to fill
__global__ void k_fill_records(uint4 *rec, uint64_t n16, uint32_t seed)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n16;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t a = mix32((uint32_t)i ^ seed), b = mix32(a + 0x9E3779B9u);
        rec[i] = make_uint4(a, b, mix32(b), mix32(a ^ b));
    }
}

__device__ __forceinline__ void load64(const uint4 *p, uint32_t (&w)[16])
{
    asm volatile("ld.global.nc.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7])
                 : "l"(p));
    asm volatile("ld.global.nc.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(w[8]), "=r"(w[9]), "=r"(w[10]), "=r"(w[11]), "=r"(w[12]), "=r"(w[13]), "=r"(w[14]), "=r"(w[15])
                 : "l"(p + 2));
}

__device__ __forceinline__ void load32(const uint4 *p, uint32_t (&w)[16])
{
    asm volatile("ld.global.nc.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7])
                 : "l"(p));
}

template <int RB>
__global__ void k_gather_probe(const uint4 *rec, uint64_t nrec, int steps, uint32_t seed, unsigned long long *sink)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t i0 = ((uint64_t)mix32(t ^ seed) * nrec) >> 32;
    uint64_t i1 = ((uint64_t)mix32(t ^ ~seed) * nrec) >> 32;
    uint32_t acc = 0;
#pragma unroll 1
    for (int s = 0; s < steps; ++s) {
        uint32_t w0[16], w1[16];
        if (RB == 64) {
            load64(rec + 4 * i0, w0);
            load64(rec + 4 * i1, w1);
        } else {
            load32(rec + 2 * i0, w0);
            load32(rec + 2 * i1, w1);
        }
        uint32_t x0 = 0, x1 = 0;
#pragma unroll
        for (int k = 0; k < RB / 4; ++k) { x0 ^= w0[k]; x1 ^= w1[k]; }
        acc += x0 + x1;
        i0 = ((uint64_t)x0 * nrec) >> 32;
        i1 = ((uint64_t)x1 * nrec) >> 32;
    }
    if (acc == 0x12345678u) atomicAdd(sink, 1ull);   // keeps the loads live
}

// The hybrid table's pattern (the dependent schedule): each step reads a 64-byte record; a share
// `ool` (out of 2^32) of the records, chosen by a hash of their contents,
// also leads to a 16-byte bucket of a second buffer (one 128-bit load,
// dependent on the record), and the next record index comes from the
// bucket.  This is the walk on rows whose alias table is out of line.
__global__ void k_gather_probe_mix(const uint4 *rec, uint64_t nrec, const uint4 *bkt, uint64_t nbkt, uint32_t ool,
                                   int steps, uint32_t seed, unsigned long long *sink)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t i0 = ((uint64_t)mix32(t ^ seed) * nrec) >> 32;
    uint64_t i1 = ((uint64_t)mix32(t ^ ~seed) * nrec) >> 32;
    uint32_t acc = 0;
#pragma unroll 1
    for (int s = 0; s < steps; ++s) {
        uint32_t w0[16], w1[16];
        load64(rec + 4 * i0, w0);
        load64(rec + 4 * i1, w1);
        uint32_t x0 = 0, x1 = 0;
#pragma unroll
        for (int k = 0; k < 16; ++k) { x0 ^= w0[k]; x1 ^= w1[k]; }
        if (mix32(x0) < ool) {
            const uint4 b = __ldg(bkt + (((uint64_t)x0 * nbkt) >> 32));
            x0 = mix32(x0 ^ b.x ^ b.y ^ b.z ^ b.w);
        }
        if (mix32(x1) < ool) {
            const uint4 b = __ldg(bkt + (((uint64_t)x1 * nbkt) >> 32));
            x1 = mix32(x1 ^ b.x ^ b.y ^ b.z ^ b.w);
        }
        acc += x0 + x1;
        i0 = ((uint64_t)x0 * nrec) >> 32;
        i1 = ((uint64_t)x1 * nrec) >> 32;
    }
    if (acc == 0x12345678u) atomicAdd(sink, 1ull);   // keeps the loads live
}

// The same pattern in the walk's split schedule: every chain issues one read
// per iteration, its next record or the bucket of the record it read last,
// so that a lane whose record has no bucket does not wait for the buckets of
// the other lanes of its warp.  Each chain makes `steps` record reads.
__global__ void k_gather_probe_mix_split(const uint4 *rec, uint64_t nrec, const uint4 *bkt, uint64_t nbkt,
                                         uint32_t ool, int steps, uint32_t seed, unsigned long long *sink)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t i0 = ((uint64_t)mix32(t ^ seed) * nrec) >> 32;
    uint64_t i1 = ((uint64_t)mix32(t ^ ~seed) * nrec) >> 32;
    uint32_t acc = 0, x0 = 0, x1 = 0;
    int n0 = 0, n1 = 0;
    bool p0 = false, p1 = false;   // the chain's next read is a bucket
#pragma unroll 1
    while (n0 < steps || n1 < steps || p0 || p1) {
        uint32_t w0[16], w1[16];
        uint4 b0 = make_uint4(0, 0, 0, 0), b1 = make_uint4(0, 0, 0, 0);
        const bool r0 = !p0 && n0 < steps, r1 = !p1 && n1 < steps;
        if (p0) b0 = __ldg(bkt + (((uint64_t)x0 * nbkt) >> 32));
        else if (r0) load64(rec + 4 * i0, w0);
        if (p1) b1 = __ldg(bkt + (((uint64_t)x1 * nbkt) >> 32));
        else if (r1) load64(rec + 4 * i1, w1);
        if (p0) {
            x0 = mix32(x0 ^ b0.x ^ b0.y ^ b0.z ^ b0.w);
            i0 = ((uint64_t)x0 * nrec) >> 32;
            acc += x0;
            p0 = false;
        } else if (r0) {
            x0 = 0;
#pragma unroll
            for (int k = 0; k < 16; ++k) x0 ^= w0[k];
            ++n0;
            if (mix32(x0) < ool) {
                p0 = true;
            } else {
                i0 = ((uint64_t)x0 * nrec) >> 32;
                acc += x0;
            }
        }
        if (p1) {
            x1 = mix32(x1 ^ b1.x ^ b1.y ^ b1.z ^ b1.w);
            i1 = ((uint64_t)x1 * nrec) >> 32;
            acc += x1;
            p1 = false;
        } else if (r1) {
            x1 = 0;
#pragma unroll
            for (int k = 0; k < 16; ++k) x1 ^= w1[k];
            ++n1;
            if (mix32(x1) < ool) {
                p1 = true;
            } else {
                i1 = ((uint64_t)x1 * nrec) >> 32;
                acc += x1;
            }
        }
    }
    if (acc == 0x12345678u) atomicAdd(sink, 1ull);   // keeps the loads live
}

}  // namespace

}  // namespace mcmi

extern "C" mcmi_status mcmi_gather_roofline(uint64_t footprint_bytes, int record_bytes, int threads_per_block,
                                            int blocks_per_sm, int steps, double *records_per_s, void *stream)
{
    using namespace mcmi;
    if (!records_per_s || footprint_bytes < 4096 || (record_bytes != 32 && record_bytes != 64) ||
        threads_per_block < 32 || threads_per_block > 1024 || blocks_per_sm < 1 || steps < 1) {
        set_error_message("mcmi_gather_roofline: bad argument");
        return MCMI_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t nrec = footprint_bytes / (uint64_t)record_bytes;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint4 *rec = nullptr;
    unsigned long long *sink = nullptr;
    cudaError_t e = cudaMallocAsync(&rec, nrec * (uint64_t)record_bytes, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&sink, 8, s);
    if (e != cudaSuccess) {
        if (rec) cudaFreeAsync(rec, s);
        set_error_message("mcmi_gather_roofline: allocation failed");
        return MCMI_ERR_OOM;
    }
    k_fill_records<<<sms * 8, 256, 0, s>>>(rec, nrec * (uint64_t)record_bytes / 16, 0x1234567u);
    const int grid = sms * blocks_per_sm;
    auto probe = record_bytes == 64 ? k_gather_probe<64> : k_gather_probe<32>;
    probe<<<grid, threads_per_block, 0, s>>>(rec, nrec, 8, 1u, sink);   // warm-up
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s);
    probe<<<grid, threads_per_block, 0, s>>>(rec, nrec, steps, 2u, sink);
    cudaEventRecord(b, s);
    e = cudaEventSynchronize(b);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFreeAsync(rec, s);
    cudaFreeAsync(sink, s);
    if (e != cudaSuccess) {
        set_error_message("mcmi_gather_roofline: kernel failed");
        return MCMI_ERR_CUDA;
    }
    *records_per_s = (double)grid * threads_per_block * 2.0 * steps / (ms * 1e-3);
    return MCMI_OK;
}

extern "C" mcmi_status mcmi_gather_roofline_mix(uint64_t record_footprint_bytes, uint64_t bucket_footprint_bytes,
                                                double bucket_share, int threads_per_block, int blocks_per_sm,
                                                int steps, double *records_per_s, void *stream)
{
    using namespace mcmi;
    if (!records_per_s || record_footprint_bytes < 4096 || bucket_footprint_bytes < 4096 ||
        !(bucket_share >= 0.0 && bucket_share <= 1.0) || threads_per_block < 32 || threads_per_block > 1024 ||
        blocks_per_sm < 1 || steps < 1) {
        set_error_message("mcmi_gather_roofline_mix: bad argument");
        return MCMI_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t nrec = record_footprint_bytes / 64, nbkt = bucket_footprint_bytes / 16;
    const uint32_t ool = bucket_share >= 1.0 ? 0xFFFFFFFFu : (uint32_t)(bucket_share * 4294967296.0);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint4 *rec = nullptr, *bkt = nullptr;
    unsigned long long *sink = nullptr;
    cudaError_t e = cudaMallocAsync(&rec, nrec * 64, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&bkt, nbkt * 16, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&sink, 8, s);
    if (e != cudaSuccess) {
        if (rec) cudaFreeAsync(rec, s);
        if (bkt) cudaFreeAsync(bkt, s);
        set_error_message("mcmi_gather_roofline_mix: allocation failed");
        return MCMI_ERR_OOM;
    }
    k_fill_records<<<sms * 8, 256, 0, s>>>(rec, nrec * 4, 0x1234567u);
    k_fill_records<<<sms * 8, 256, 0, s>>>(bkt, nbkt, 0x7654321u);
    const int grid = sms * blocks_per_sm;
    // both schedules (every chain waits for its bucket within the step, or
    // reads it in the next iteration); the faster one is the ceiling
    k_gather_probe_mix<<<grid, threads_per_block, 0, s>>>(rec, nrec, bkt, nbkt, ool, 8, 1u, sink);   // warm-up
    k_gather_probe_mix_split<<<grid, threads_per_block, 0, s>>>(rec, nrec, bkt, nbkt, ool, 8, 1u, sink);
    cudaEvent_t a, b, c;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventCreate(&c);
    cudaEventRecord(a, s);
    k_gather_probe_mix<<<grid, threads_per_block, 0, s>>>(rec, nrec, bkt, nbkt, ool, steps, 2u, sink);
    cudaEventRecord(b, s);
    k_gather_probe_mix_split<<<grid, threads_per_block, 0, s>>>(rec, nrec, bkt, nbkt, ool, steps, 3u, sink);
    cudaEventRecord(c, s);
    e = cudaEventSynchronize(c);
    float ms = 0.0f, ms_split = 0.0f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventElapsedTime(&ms_split, b, c);
    if (ms_split > 0.0f && ms_split < ms) ms = ms_split;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaEventDestroy(c);
    cudaFreeAsync(rec, s);
    cudaFreeAsync(bkt, s);
    cudaFreeAsync(sink, s);
    if (e != cudaSuccess) {
        set_error_message("mcmi_gather_roofline_mix: kernel failed");
        return MCMI_ERR_CUDA;
    }
    *records_per_s = (double)grid * threads_per_block * 2.0 * steps / (ms * 1e-3);
    return MCMI_OK;
}
