// Peak microbenchmarks for the rooflines of the LSHBloom kernels on one GPU.
//
//  * random sector gathers: 4-byte loads at random 32-byte sectors of a
//    buffer far larger than L2, in several load forms (the Bloom probe's
//    access pattern), a full 32-byte sector read by 8 lanes (the blocked
//    layout's pattern), and random 4-byte atomic ORs (the insert's pattern);
//  * instruction issue rates: 32x32->64 multiply-adds (mad.wide.u32), 32-bit
//    multiply-adds, and ALU operations (min, add, 3-input xor, funnel shift);
//  * the signature stage's own ceiling: the library's SHA-1 window hash and
//    its MinHash fold (sig_kernels.cuh), run from registers and shared memory
//    with no global traffic, alone and together.
// Each entry point launches on the legacy default stream, brackets the
// launch with CUDA events and returns the elapsed milliseconds.
#include <cuda_runtime.h>

#include <cstdint>

#include "sig_kernels.cuh"

#define MB_API extern "C" __attribute__((visibility("default")))

namespace {

__device__ uint32_t g_sink[1024];

__device__ __forceinline__ uint64_t mb_mix(uint64_t z) {
    z = (z ^ (z >> 33)) * 0xff51afd7ed558ccdull;
    return z ^ (z >> 29);
}

template <int MODE>
__device__ __forceinline__ uint32_t mb_load(const uint32_t *p) {
    uint32_t v;
    if constexpr (MODE == 0) asm volatile("ld.global.nc.u32 %0, [%1];" : "=r"(v) : "l"(p));
    else if constexpr (MODE == 1) asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(v) : "l"(p));
    else if constexpr (MODE == 2) asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p));
    else if constexpr (MODE == 3) asm volatile("ld.global.nc.L2::64B.u32 %0, [%1];" : "=r"(v) : "l"(p));
    else if constexpr (MODE == 4) asm volatile("ld.global.cv.u32 %0, [%1];" : "=r"(v) : "l"(p));
    else asm volatile("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// MODE 0-5: per_thread random 4-byte loads (one per random sector), eight in
// flight per thread.  MODE 6: random atomic ORs.  MODE 7: groups of 8 lanes
// read the 8 words of one random sector.
template <int MODE>
__global__ void __launch_bounds__(256) k_gather(uint32_t *buf, uint64_t sect_mask,
                                                uint64_t per_thread, uint64_t seed) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    if constexpr (MODE == 7) {
        const uint32_t lane8 = threadIdx.x & 7;
        const uint64_t grp = tid >> 3;
        for (uint64_t i = 0; i < per_thread; i += 8) {
            uint32_t v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint64_t s = mb_mix(seed + grp * 0x9e3779b97f4a7c15ull + i + u) & sect_mask;
                v[u] = __ldg(buf + s * 8 + lane8);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) acc ^= v[u];
        }
    } else {
        for (uint64_t i = 0; i < per_thread; i += 8) {
            uint32_t v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint64_t r = mb_mix(seed + tid * 0x9e3779b97f4a7c15ull + i + u);
                uint32_t *p = buf + (r & sect_mask) * 8 + ((r >> 59) & 7);
                if constexpr (MODE == 6) {
                    atomicOr(p, 1u << ((r >> 40) & 31));
                    v[u] = 0;
                } else {
                    v[u] = mb_load<MODE>(p);
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) acc ^= v[u];
        }
    }
    if (acc == 0x9e3779b9u) g_sink[tid & 1023] = acc;
}

// KIND 0 mad.wide.u32, 1 mad.lo.u32, 2 min.u32, 3 add.u32, 4 3-input xor,
// 5 funnel shift: eight independent chains per thread.
template <int KIND>
__global__ void __launch_bounds__(256) k_issue(uint64_t iters) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t w[8];
    uint32_t r[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        w[i] = t * 0x9e3779b97f4a7c15ull + i;
        r[i] = t * 2654435761u + i * 40503u;
    }
    const uint32_t x = t | 1u, y = t ^ 0x5bd1e995u;
    for (uint64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if constexpr (KIND == 0) asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(w[i]) : "r"(x + i), "r"(y));
            else if constexpr (KIND == 1) asm volatile("mad.lo.u32 %0, %1, %2, %0;" : "+r"(r[i]) : "r"(x + i), "r"(y));
            else if constexpr (KIND == 2) asm volatile("min.u32 %0, %0, %1;" : "+r"(r[i]) : "r"(x + i));
            else if constexpr (KIND == 3) asm volatile("add.u32 %0, %0, %1;" : "+r"(r[i]) : "r"(x + i));
            else if constexpr (KIND == 4) asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(r[i]) : "r"(x + i), "r"(y));
            else asm volatile("shf.r.wrap.b32 %0, %0, %1, %2;" : "+r"(r[i]) : "r"(x + i), "r"(y));
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) acc ^= r[i] ^ (uint32_t)w[i] ^ (uint32_t)(w[i] >> 32);
    if (acc == 0x9e3779b9u) g_sink[t & 1023] = acc;
}

// The signature stage's arithmetic without memory: KIND 0 the MinHash fold of
// 32 hashes from a shared slot into PPL minima per lane (as fold_pass does per
// 32-shingle step), KIND 1 the 32 SHA-1 window hashes of a step (as
// window_hash_regs computes them), KIND 2 both.
template <int KIND>
__global__ void __launch_bounds__(lshb::kSigThreads) k_ceiling(uint64_t steps,
                                                               const __grid_constant__ lshb::PermSlice c) {
    __shared__ uint4 hb[lshb::kSigThreads / 32][8];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    lshb::LaneCoef<4> cf;
    cf.load(c, 121, lane);
    uint32_t mn[4] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu};
    uint32_t guard = 0, acc = 0;
    uint32_t ta = (blockIdx.x * 64 + threadIdx.x) * 2654435761u, tb = ta ^ 0x85ebca6bu;
    uint32_t *hbuf = reinterpret_cast<uint32_t *>(hb[wib]);
    hbuf[lane] = ta * 0x27d4eb2fu;
    __syncwarp();
    for (uint64_t s = 0; s < steps; ++s) {
        if constexpr (KIND != 0) {
            const uint32_t h = lshb::window_hash_regs<5>(ta, tb, lane);
            ta = tb;
            tb = h;
            acc ^= h;
            if constexpr (KIND == 2) {
                __syncwarp();
                hbuf[lane] = h;
                __syncwarp();
            }
        } else {
            __syncwarp();
            hbuf[lane] += 0x9e3779b9u;
            __syncwarp();
        }
        if constexpr (KIND != 1) {
            const uint4 *hv4 = reinterpret_cast<const uint4 *>(hbuf);
#pragma unroll 1
            for (int g = 0; g < 8; ++g) lshb::fold4<4, true>(mn, cf, hv4[g], guard);
        }
    }
    acc ^= mn[0] ^ mn[1] ^ mn[2] ^ mn[3] ^ guard;
    if (acc == 0x9e3779b9u) g_sink[threadIdx.x] = acc;
}

template <typename F>
float timed(F launch) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, 0);
    launch();
    cudaEventRecord(e1, 0);
    cudaEventSynchronize(e1);
    float ms = -1.f;
    if (cudaGetLastError() == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

}  // namespace

// Random-sector gather over buf (sect_mask + 1 sectors of 32 bytes, a power
// of two; the caller owns the buffer).  threads * per_thread accesses
// (per_thread a multiple of 8).  Returns elapsed ms, < 0 on a CUDA error.
MB_API float mb_gather(void *buf, uint64_t sect_mask, uint64_t threads, uint64_t per_thread,
                       int mode, uint64_t seed) {
    const unsigned grid = (unsigned)((threads + 255) / 256);
    uint32_t *b = (uint32_t *)buf;
    return timed([&] {
        switch (mode) {
            case 0: k_gather<0><<<grid, 256>>>(b, sect_mask, per_thread, seed); break;
            case 1: k_gather<1><<<grid, 256>>>(b, sect_mask, per_thread, seed); break;
            case 2: k_gather<2><<<grid, 256>>>(b, sect_mask, per_thread, seed); break;
            case 3: k_gather<3><<<grid, 256>>>(b, sect_mask, per_thread, seed); break;
            case 4: k_gather<4><<<grid, 256>>>(b, sect_mask, per_thread, seed); break;
            case 5: k_gather<5><<<grid, 256>>>(b, sect_mask, per_thread, seed); break;
            case 6: k_gather<6><<<grid, 256>>>(b, sect_mask, per_thread, seed); break;
            default: k_gather<7><<<grid, 256>>>(b, sect_mask, per_thread, seed); break;
        }
    });
}

// Issue rate of one instruction kind: blocks x 256 threads x iters x 8 ops.
MB_API float mb_issue(int kind, uint64_t blocks, uint64_t iters) {
    const unsigned g = (unsigned)blocks;
    return timed([&] {
        switch (kind) {
            case 0: k_issue<0><<<g, 256>>>(iters); break;
            case 1: k_issue<1><<<g, 256>>>(iters); break;
            case 2: k_issue<2><<<g, 256>>>(iters); break;
            case 3: k_issue<3><<<g, 256>>>(iters); break;
            case 4: k_issue<4><<<g, 256>>>(iters); break;
            default: k_issue<5><<<g, 256>>>(iters); break;
        }
    });
}

// Signature-stage ceiling: blocks x 2 warps x steps 32-shingle steps, P = 121
// (coefficients from host arrays a, b of 121 entries).
MB_API float mb_ceiling(int kind, uint64_t blocks, uint64_t steps, const uint64_t *a,
                        const uint64_t *b) {
    lshb::PermSlice c;
    for (int i = 0; i < lshb::kMaxPC; ++i) {
        const uint64_t ai = i < 121 ? a[i] : 0, bi = i < 121 ? b[i] : 0;
        c.a0[i] = (uint32_t)ai;
        c.a1[i] = (uint32_t)(ai >> 32);
        c.b0[i] = (uint32_t)bi;
        c.b1[i] = (uint32_t)(bi >> 32);
    }
    const unsigned g = (unsigned)blocks;
    return timed([&] {
        switch (kind) {
            case 0: k_ceiling<0><<<g, lshb::kSigThreads>>>(steps, c); break;
            case 1: k_ceiling<1><<<g, lshb::kSigThreads>>>(steps, c); break;
            default: k_ceiling<2><<<g, lshb::kSigThreads>>>(steps, c); break;
        }
    });
}

// Resident blocks per SM of the ceiling kernel (for sizing its grid).
MB_API int mb_ceiling_occupancy(int kind) {
    int nb = 0;
    if (kind == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_ceiling<0>, lshb::kSigThreads, 0);
    else if (kind == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_ceiling<1>, lshb::kSigThreads, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_ceiling<2>, lshb::kSigThreads, 0);
    return nb;
}
