// Device helpers shared by the fused step kernels (tslb_step.cu,
// tslb_step_ce.cu): ghost resolution, the inlet state, cp.async, the storage
// conversions, packed FP32 arithmetic on a pair of nodes, the D1Q3 sweep
// pieces, and the interface stencil of the phase field.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tslb_internal.h"

namespace tslb {
namespace {

constexpr unsigned FULL = 0xffffffffu;
// Interior columns of a tile: lanes 1 .. 28 of a warp; lanes 0 and 29 stage
// the halo columns, lanes 30 and 31 are spare (the stencils take neighbour
// columns from neighbour lanes, lane 31 standing in for the column left of
// lane 0).
constexpr int TX = 28;
constexpr int PHX = 34;       // footprint columns of a tile: x0 - 2 .. x0 + 31

// ------------------------------------------------------------------ helpers

// Source coordinate of grid coordinate g on an axis of n nodes whose lower /
// upper faces follow rule lo / hi.  sign = -1 for a mirror image, inlet = 1
// for the inlet ghost.  Coordinates farther out than any stencil reaches are
// clamped into the grid (their values are never used).  A HALO face (z only)
// maps its ghost planes -2, -1 / n, n + 1 to the planes stored after the
// interior (n + 2, n + 3 / n, n + 1).
__device__ __forceinline__ int resolve_axis(int g, int n, int lo, int hi, float& sign, int& inlet) {
    sign = 1.f;
    if (g >= 0 && g < n) return g;
    const int kind = g < 0 ? lo : hi;
    if (kind == BC_HALO) return g < 0 ? max(n + kHaloPlanes + g, n + 2) : min(g, n + 1);
    int s;
    if (kind == BC_PERIODIC) {
        s = g % n;
        if (s < 0) s += n;
    } else if (kind == BC_FREE_SLIP) {
        sign = -1.f;
        s = g < 0 ? -1 - g : 2 * n - 1 - g;
    } else {
        if (kind == BC_INLET) inlet = 1;
        s = g < 0 ? 0 : n - 1;
    }
    return min(max(s, 0), n - 1);
}

// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11).
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

// Imposed phase field of the inlet at lateral node (x, y): smoothed top hat.
__device__ __forceinline__ float inlet_phi(const StepParams& P, int x, int y) {
    const float dx = (float)x - P.inlet_cx, dy = (float)y - P.inlet_cy;
    const float r = sqrtf(dx * dx + dy * dy);
    return -tanhf((r - P.inlet_half_d) * P.inlet_two_over_w);
}

// Imposed inlet velocity at (x, y) and step t: s (U + xi), s = (1 + phi_B)/2,
// xi_c = a |U| (2 r_c - 1), r_c from Philox on counter (x + nx y, t_lo, t_hi, 0).
__device__ void inlet_velocity(const StepParams& P, int x, int y, long long t, float u[3]) {
    const float s = 0.5f * (1.f + inlet_phi(P, x, y));
    uint32_t c[4] = {(uint32_t)(x + P.nx * y), (uint32_t)((unsigned long long)t & 0xffffffffu),
                     (uint32_t)((unsigned long long)t >> 32), 0u};
    philox4x32_10(c, P.seed_lo, P.seed_hi);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float rc = (float)(c[k] >> 8) * (1.f / 16777216.f);
        const float xi = P.noise_amp * P.inlet_umag * (2.f * rc - 1.f);
        u[k] = s * (P.inlet_u[k] + xi);
    }
}

__device__ __forceinline__ void cp_async4(float* smem_dst, const float* gmem_src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ------------------------------------------------- TMA tile loads (sm_90+)

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// Makes mbarrier initialisation visible to the async (TMA) proxy.
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
// Orders this thread's view of shared memory (generic proxy) before its
// subsequent bulk copies (async proxy) into the same memory.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
// Orders this thread's later TMA uses of the tensor maps at `m` (device
// memory, written before the launch) after their generic-proxy contents.
template <typename T>
__device__ __forceinline__ void fence_tensormap_acquire(const T* m) {
    constexpr int n = (int)(sizeof(T) / 128);
#pragma unroll
    for (int k = 0; k < n; ++k)
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;\n" ::"l"(
                         reinterpret_cast<const char*>(m) + 128 * k)
                     : "memory");
}
// Bounded wait for the completion of phase `parity` of an mbarrier: gives up
// (returns false) after about kWaitCycles SM cycles (~1 s) instead of spinning
// forever if the copies it counts never arrive.
constexpr long long kWaitCycles = 2000000000LL;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitCycles) return false;
    return true;
}
// Tiled bulk tensor copies global -> shared memory, completing on `bar`.
// Coordinates are element indices, innermost first; the innermost one must
// be a multiple of 16 bytes (the callers align it down).
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int x, int y, int z, int f,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(f), "r"(smem_u32(bar))
        : "memory");
}

// Tiled bulk tensor copy shared -> global memory (4D), in the calling
// thread's bulk async-group; elements outside the tensor are not written.
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, const void* src, int x, int y, int z, int f) {
    asm volatile(
        "cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4, %5}], [%1];\n" ::"l"(
            reinterpret_cast<unsigned long long>(map)),
        "r"(smem_u32(src)), "r"(x), "r"(y), "r"(z), "r"(f)
        : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
// Waits until at most N bulk groups of this thread still read shared memory.
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;\n" ::"n"(N) : "memory");
}
// Waits until at most N bulk groups of this thread are still in flight.
template <int N>
__device__ __forceinline__ void bulk_wait() {
    asm volatile("cp.async.bulk.wait_group %0;\n" ::"n"(N) : "memory");
}

// ------------------------------------------ tensor memory (tcgen05, sm_100+)
//
// The step kernels of 14 and 16 warps keep per-thread state of the z march in
// tensor memory (TMEM) instead of registers between planes: the block
// allocates TMEM columns once, each warp reaches the 32 TMEM lanes of its
// quarter (warp w: lanes 32 (w % 4) .. 32 (w % 4) + 31) through 32x32b
// loads and stores (thread t of the warp <-> lane 32 (w % 4) + t, one 32-bit
// value per column), and the block frees the columns before it exits.

// Allocates ncols TMEM columns (a power of two >= 32) for the block; the
// column address is written to *dst (shared memory).  All threads of one warp.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
}
// Frees the columns of tmem_alloc.  All threads of the allocating warp, after
// every TMEM access of the block has completed.
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}
// Orders TMEM operations before / after a thread synchronisation (bar.sync).
__device__ __forceinline__ void tmem_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
// Eight consecutive columns of this thread's lane, from / to registers.
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float* v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};\n" ::"r"(taddr), "f"(v[0]),
        "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
        : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
                 : "r"(taddr)
                 : "memory");
}
// Waits for this thread's TMEM loads; the loaded registers are operands so
// that no use of them is placed before the wait.
__device__ __forceinline__ void tmem_wait_ld(float (&v)[40]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;\n"
                 : "+f"(v[0]), "+f"(v[1]), "+f"(v[2]), "+f"(v[3]), "+f"(v[4]), "+f"(v[5]), "+f"(v[6]), "+f"(v[7]),
                   "+f"(v[8]), "+f"(v[9]), "+f"(v[10]), "+f"(v[11]), "+f"(v[12]), "+f"(v[13]), "+f"(v[14]),
                   "+f"(v[15]), "+f"(v[16]), "+f"(v[17]), "+f"(v[18]), "+f"(v[19])
                 :
                 : "memory");
    asm volatile(""
                 : "+f"(v[20]), "+f"(v[21]), "+f"(v[22]), "+f"(v[23]), "+f"(v[24]), "+f"(v[25]), "+f"(v[26]),
                   "+f"(v[27]), "+f"(v[28]), "+f"(v[29]), "+f"(v[30]), "+f"(v[31]), "+f"(v[32]), "+f"(v[33]),
                   "+f"(v[34]), "+f"(v[35]), "+f"(v[36]), "+f"(v[37]), "+f"(v[38]), "+f"(v[39])
                 :
                 : "memory");
}
// The same for 48 values.
__device__ __forceinline__ void tmem_wait_ld48(float (&v)[48]) {
    tmem_wait_ld(reinterpret_cast<float(&)[40]>(v));
    asm volatile(""
                 : "+f"(v[40]), "+f"(v[41]), "+f"(v[42]), "+f"(v[43]), "+f"(v[44]), "+f"(v[45]), "+f"(v[46]),
                   "+f"(v[47])
                 :
                 : "memory");
}
// Waits for this thread's TMEM stores (their source registers may then be reused).
__device__ __forceinline__ void tmem_wait_st(const float (&v)[40]) {
    asm volatile("tcgen05.wait::st.sync.aligned;\n" ::"f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]),
                 "f"(v[5]), "f"(v[6]), "f"(v[7]), "f"(v[8]), "f"(v[9]), "f"(v[10]), "f"(v[11]), "f"(v[12]),
                 "f"(v[13]), "f"(v[14]), "f"(v[15]), "f"(v[16]), "f"(v[17]), "f"(v[18]), "f"(v[19])
                 : "memory");
    asm volatile("" ::"f"(v[20]), "f"(v[21]), "f"(v[22]), "f"(v[23]), "f"(v[24]), "f"(v[25]), "f"(v[26]),
                 "f"(v[27]), "f"(v[28]), "f"(v[29]), "f"(v[30]), "f"(v[31]), "f"(v[32]), "f"(v[33]), "f"(v[34]),
                 "f"(v[35]), "f"(v[36]), "f"(v[37]), "f"(v[38]), "f"(v[39])
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_st48(const float (&v)[48]) {
    tmem_wait_st(reinterpret_cast<const float(&)[40]>(v));
    asm volatile("" ::"f"(v[40]), "f"(v[41]), "f"(v[42]), "f"(v[43]), "f"(v[44]), "f"(v[45]), "f"(v[46]),
                 "f"(v[47])
                 : "memory");
}

// Stored <-> FP32 conversion of one field value.  16-bit storage keeps
// scaled deviations from the rest state (rho - 1, u, P and the phase field's
// deviation below); FP32 storage keeps the values themselves.
//
// The phase field in 16-bit storage.  Its bulk values sit near +-1, where a
// 16-bit float is coarsest (2^-11 in FP16, 2^-8 in BF16 below 1), and the
// rounding of the bulk then moves the interfaces.  So it is stored as the
// deviation from the nearer of +-(1 + m), m = 1/16:
//   d = phi - (1 + m) for phi >= 0 (d < 0),  d = phi + (1 + m) for phi < 0 (d > 0),
// which is small in the bulk (|d| ~ m, resolved to 2^-15 in FP16) and whose
// sign tells the branch back: phi = d - copysign(1 + m, d).  The margin m
// leaves room for the overshoot of +-1 the phase field shows at interfaces
// (a few 10^-3); beyond it, |phi| would saturate at 1 + m (d rounds to -0 /
// +0, which decode to +-(1 + m)).
constexpr float kPhiOff = 1.f + 1.f / 16.f;
__device__ __forceinline__ float phi_encode(float v) {
    const float d = v - copysignf(kPhiOff, v);
    return signbit(v) ? (d > 0.f ? d : 0.f) : (d < 0.f ? d : -0.f);
}
__device__ __forceinline__ float phi_decode(float d) { return d - copysignf(kPhiOff, d); }

template <typename S>
struct Io;
template <>
struct Io<float> {
    static constexpr bool kAsync = true;
    static __device__ __forceinline__ float from_raw(unsigned short, float) { return 0.f; }
    static __device__ __forceinline__ float cvt(float v, float) { return v; }
    static __device__ __forceinline__ float ld(const float* p, float) { return __ldg(p); }
    static __device__ __forceinline__ void st(float* p, float v, float) { *p = v; }
    static __device__ __forceinline__ float round_trip(float v, float, float) { return v; }
    // the phase field (FP32: the value itself)
    static __device__ __forceinline__ float from_raw_phi(unsigned short, float) { return 0.f; }
    static __device__ __forceinline__ float cvt_phi(float v, float) { return v; }
    static __device__ __forceinline__ float ld_phi(const float* p, float) { return __ldg(p); }
    static __device__ __forceinline__ void st_phi(float* p, float v, float) { *p = v; }
    static __device__ __forceinline__ float round_trip_phi(float v, float, float) { return v; }
};
template <>
struct Io<__half> {
    static constexpr bool kAsync = false;
    static __device__ __forceinline__ float from_raw(unsigned short r, float inv) {
        return __half2float(__ushort_as_half(r)) * inv;
    }
    static __device__ __forceinline__ float cvt(__half v, float inv) { return __half2float(v) * inv; }
    static __device__ __forceinline__ float ld(const __half* p, float inv) { return __half2float(__ldg(p)) * inv; }
    static __device__ __forceinline__ void st(__half* p, float v, float s) { *p = __float2half_rn(v * s); }
    static __device__ __forceinline__ float round_trip(float v, float s, float inv) {
        return __half2float(__float2half_rn(v * s)) * inv;
    }
    static __device__ __forceinline__ float from_raw_phi(unsigned short r, float inv) {
        return phi_decode(from_raw(r, inv));
    }
    static __device__ __forceinline__ float cvt_phi(__half v, float inv) { return phi_decode(cvt(v, inv)); }
    static __device__ __forceinline__ float ld_phi(const __half* p, float inv) { return phi_decode(ld(p, inv)); }
    static __device__ __forceinline__ void st_phi(__half* p, float v, float s) { st(p, phi_encode(v), s); }
    static __device__ __forceinline__ float round_trip_phi(float v, float s, float inv) {
        return phi_decode(round_trip(phi_encode(v), s, inv));
    }
};
template <>
struct Io<__nv_bfloat16> {
    static constexpr bool kAsync = false;
    static __device__ __forceinline__ float from_raw(unsigned short r, float inv) {
        return __bfloat162float(__ushort_as_bfloat16(r)) * inv;
    }
    static __device__ __forceinline__ float cvt(__nv_bfloat16 v, float inv) { return __bfloat162float(v) * inv; }
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p, float inv) {
        return __bfloat162float(__ldg(p)) * inv;
    }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, float v, float s) { *p = __float2bfloat16_rn(v * s); }
    static __device__ __forceinline__ float round_trip(float v, float s, float inv) {
        return __bfloat162float(__float2bfloat16_rn(v * s)) * inv;
    }
    static __device__ __forceinline__ float from_raw_phi(unsigned short r, float inv) {
        return phi_decode(from_raw(r, inv));
    }
    static __device__ __forceinline__ float cvt_phi(__nv_bfloat16 v, float inv) { return phi_decode(cvt(v, inv)); }
    static __device__ __forceinline__ float ld_phi(const __nv_bfloat16* p, float inv) {
        return phi_decode(ld(p, inv));
    }
    static __device__ __forceinline__ void st_phi(__nv_bfloat16* p, float v, float s) { st(p, phi_encode(v), s); }
    static __device__ __forceinline__ float round_trip_phi(float v, float s, float inv) {
        return phi_decode(round_trip(phi_encode(v), s, inv));
    }
};

// ------------------------------------------------------- packed FP32 helpers

// Two lattice nodes per thread (rows 2w and 2w+1 of the tile) are processed
// together with the packed FP32 instructions of sm_100+ (one instruction, two
// lanes of arithmetic): .x is the node of row 2w, .y the node of row 2w+1.
__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return __fadd2_rn(a, b); }
// (packed subtraction: PTX sub.rn.f32x2; an FMA by -1 would hold a constant
// pair in registers and take the FMA form of the instruction)
__device__ __forceinline__ float2 operator-(float2 a, float2 b) {
    float2 d;
    asm("{\n"
        " .reg .b64 ra, rb, rd;\n"
        " mov.b64 ra, {%2, %3};\n"
        " mov.b64 rb, {%4, %5};\n"
        " sub.rn.f32x2 rd, ra, rb;\n"
        " mov.b64 {%0, %1}, rd;\n"
        "}\n"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 operator*(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 operator*(float s, float2 b) { return __fmul2_rn(make_float2(s, s), b); }
__device__ __forceinline__ float2 mad(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mad(float s, float2 b, float2 c) { return __ffma2_rn(make_float2(s, s), b, c); }
__device__ __forceinline__ float2 bc(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 rcp2(float2 a) { return make_float2(__fdividef(1.f, a.x), __fdividef(1.f, a.y)); }
__device__ __forceinline__ float2 shfl_up2(float2 v) {
    return make_float2(__shfl_up_sync(FULL, v.x, 1), __shfl_up_sync(FULL, v.y, 1));
}
__device__ __forceinline__ float2 shfl_down2(float2 v) {
    return make_float2(__shfl_down_sync(FULL, v.x, 1), __shfl_down_sync(FULL, v.y, 1));
}

// One axis of the streaming sweep.  (k0, k1, k2) are the Hermite coefficients
// of the axis (k2 pre-multiplied by h2(+-1) = 2/3); the unnormalised 1D
// populations (x 6) are
//   p(-1) = k0 - k1 + k2,   p(0) = 4 k0 - 2 k2,   p(+1) = k0 + k1 + k2,
// and after the shift the raw moments of the axis are
//   M0 = q- + q0 + q+,   M1 = q+ - q-,   M2 = q+ + q-.
struct Tri2 {
    float2 m, z, p;
};
__device__ __forceinline__ Tri2 pops2(float2 k0, float2 k1, float2 k2) {
    const float2 s = k0 + k2;
    return {s - k1, mad(4.f, k0, -2.f * k2), s + k1};
}
// ... for k2 = 0
__device__ __forceinline__ Tri2 pops2_01(float2 k0, float2 k1) { return {k0 - k1, 4.f * k0, k0 + k1}; }
// x sweep of two nodes: shifts along the warp (lanes = x), then x moments;
// the rest population 4 k0 - 2 k2 is folded into M0 (it is not shifted).
__device__ __forceinline__ void xsweep2(float2 k0, float2 k1, float2 k2, float2& m0, float2& m1, float2& m2) {
    const float2 s0 = k0 + k2;
    const float2 qp = shfl_up2(s0 + k1), qm = shfl_down2(s0 - k1);
    const float2 s = qp + qm;
    m0 = mad(4.f, k0, mad(-2.f, k2, s));
    m1 = qp - qm;
    m2 = s;
}
// ... for k2 = 0
__device__ __forceinline__ void xsweep2_01(float2 k0, float2 k1, float2& m0, float2& m1, float2& m2) {
    const float2 qp = shfl_up2(k0 + k1), qm = shfl_down2(k0 - k1);
    const float2 s = qp + qm;
    m0 = mad(4.f, k0, s);
    m1 = qp - qm;
    m2 = s;
}
// ... for k1 = k2 = 0
__device__ __forceinline__ void xsweep2_0(float2 k0, float2& m0, float2& m1, float2& m2) {
    const float2 qp = shfl_up2(k0), qm = shfl_down2(k0);
    const float2 s = qp + qm;
    m0 = mad(4.f, k0, s);
    m1 = qp - qm;
    m2 = s;
}
__device__ __forceinline__ float2 s0v(float2 a, float2 b, float2 c) { return mad(4.f, b, a + c); }
__device__ __forceinline__ float2 l2v(float2 a, float2 b, float2 c) { return mad(-2.f, b, a + c); }

// Interface terms of a node pair from the y combinations of the phase field
// at the columns x - 1, x, x + 1 (index 0, 1, 2): S = 4 c + (c(+1) + c(-1)),
// D = c(+1) - c(-1), L = (c(+1) + c(-1)) - 2 c, applied along y to the z
// combinations {S, D, L} (yS = S_y S_z, yDS = D_y S_z, yLS = L_y S_z,
// ySD = S_y D_z, yDD = D_y D_z, ySL = S_y L_z).  The isotropic D3Q27 stencils
// are kept unscaled: G = 72 grad phi, Hd = 36 H_aa, Ho = 24 H_ab.  Then the
// regularised normal n = grad phi / sqrt(|grad phi|^2 + eps^2) = G / |G|_eps
// (eps scaled by 72), the curvature kappa = div n = (tr H - n.H.n) / |grad phi|
// and the CSF force F = -(sigma/2) kappa grad phi (Sec. 2.2) become
//   F = (sig_half / 36) (tr Hd - G.H'.G / |G|^2) / |G| * G,
// where sig_half = -sigma/2 and H' weighs the off-diagonal terms 2 * 36 / 24.
// keep = 0 gives F = n = 0 (a node that carries no interface terms), keep = 1
// the terms above.
__device__ __forceinline__ void interface_x(const float2 (&yS)[3], const float2 (&yDS)[3], const float2 (&yLS)[3],
                                            const float2 (&ySD)[3], const float2 (&yDD)[3], const float2 (&ySL)[3],
                                            float sig_half, float eps2, float2& Fx, float2& Fy, float2& Fz,
                                            float2& nxv, float2& nyv, float2& nzv, float keep = 1.f) {
    const float2 gx = yS[2] - yS[0];
    const float2 gy = s0v(yDS[0], yDS[1], yDS[2]);
    const float2 gz = s0v(ySD[0], ySD[1], ySD[2]);
    const float2 hxx = l2v(yS[0], yS[1], yS[2]);
    const float2 hyy = s0v(yLS[0], yLS[1], yLS[2]);
    const float2 hzz = s0v(ySL[0], ySL[1], ySL[2]);
    const float2 hxy = yDS[2] - yDS[0];
    const float2 hxz = ySD[2] - ySD[0];
    const float2 hyz = s0v(yDD[0], yDD[1], yDD[2]);

    const float2 m2 = mad(gx, gx, mad(gy, gy, mad(gz, gz, bc(72.f * 72.f * eps2))));
    // (with eps = 0 a node without gradient has G = 0: the floor keeps im finite, so n = F = 0)
    const float2 im = keep * make_float2(rsqrtf(fmaxf(m2.x, 1e-30f)), rsqrtf(fmaxf(m2.y, 1e-30f)));
    nxv = gx * im;
    nyv = gy * im;
    nzv = gz * im;
    const float2 ghg = mad(gx, mad(gx, hxx, 3.f * mad(gy, hxy, gz * hxz)),
                           mad(gy, mad(gy, hyy, 3.f * (gz * hyz)), gz * gz * hzz));
    const float2 fk = ((sig_half * (1.f / 36.f)) * im) * ((hxx + hyy + hzz) - ghg * (im * im));
    Fx = fk * gx;
    Fy = fk * gy;
    Fz = fk * gz;
}

// The six y combinations of one phase-field column for the row pair, from
// the z combinations {S, D, L} of rows 2w .. 2w+3 (scalar arithmetic: the
// operands come from four different rows, packing them would cost moves).
__device__ __forceinline__ void ycomb(const float (&zS)[4], const float (&zD)[4], const float (&zL)[4], float2& yS,
                                      float2& yDS, float2& yLS, float2& ySD, float2& yDD, float2& ySL) {
    yS = make_float2(fmaf(4.f, zS[1], zS[0] + zS[2]), fmaf(4.f, zS[2], zS[1] + zS[3]));
    yDS = make_float2(zS[2] - zS[0], zS[3] - zS[1]);
    yLS = make_float2(fmaf(-2.f, zS[1], zS[0] + zS[2]), fmaf(-2.f, zS[2], zS[1] + zS[3]));
    ySD = make_float2(fmaf(4.f, zD[1], zD[0] + zD[2]), fmaf(4.f, zD[2], zD[1] + zD[3]));
    yDD = make_float2(zD[2] - zD[0], zD[3] - zD[1]);
    ySL = make_float2(fmaf(4.f, zL[1], zL[0] + zL[2]), fmaf(4.f, zL[2], zL[1] + zL[3]));
}

// Interface terms of the staged row pair from the z combinations {S, D, L}
// of rows 2w .. 2w+3 of the lane's own footprint column (lane 31: column 0):
// y combinations of that column, those of the columns x -+ 1 from the
// neighbour lanes (a third of the loads and y arithmetic of forming all three
// columns in every lane, for 24 shuffles), then interface_x.  Valid in lanes
// 0 .. 29 (the staged columns of a 28-column tile).
__device__ __forceinline__ void interface_nb(const float (&zS)[4], const float (&zD)[4], const float (&zL)[4],
                                             int lane, float sig_half, float eps2, float2& Fx, float2& Fy,
                                             float2& Fz, float2& nxv, float2& nyv, float2& nzv, float keep = 1.f) {
    float2 yS[3], yDS[3], yLS[3], ySD[3], yDD[3], ySL[3];
    ycomb(zS, zD, zL, yS[1], yDS[1], yLS[1], ySD[1], yDD[1], ySL[1]);
    const int left = (lane + 31) & 31;
    auto nb = [&](float2 (&y)[3]) {
        y[0] = make_float2(__shfl_sync(FULL, y[1].x, left), __shfl_sync(FULL, y[1].y, left));
        y[2] = shfl_down2(y[1]);
    };
    nb(yS);
    nb(yDS);
    nb(yLS);
    nb(ySD);
    nb(yDD);
    nb(ySL);
    interface_x(yS, yDS, yLS, ySD, yDD, ySL, sig_half, eps2, Fx, Fy, Fz, nxv, nyv, nzv, keep);
}

// Footprint column a lane forms its stencil values for: its own staged column
// (footprint column lane + 1), lane 31 the column left of lane 0's.
__device__ __forceinline__ int own_column(int lane) { return lane == 31 ? 0 : lane + 1; }

// Interface terms of the staged row pair (tile rows 2w and 2w+1; .x / .y)
// from z combinations stored as three planes of the footprint
// ([3][NPH]: phi, phi(z+1) + phi(z-1), phi(z+1) - phi(z-1)).
template <int NPH>
__device__ __forceinline__ void interface2(const float* zb, int lane, int w, float sig_half, float eps2,
                                           float2& phi, float2& Fx, float2& Fy, float2& Fz, float2& nxv,
                                           float2& nyv, float2& nzv) {
    float zS[4], zD[4], zL[4];
    const int col = own_column(lane);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int e = col + PHX * (2 * w + r);
        const float c0 = zb[e], c1 = zb[NPH + e], c2 = zb[2 * NPH + e];
        zS[r] = fmaf(4.f, c0, c1);
        zD[r] = c2;
        zL[r] = fmaf(-2.f, c0, c1);
        if (r == 1) phi.x = c0;
        if (r == 2) phi.y = c0;
    }
    interface_nb(zS, zD, zL, lane, sig_half, eps2, Fx, Fy, Fz, nxv, nyv, nzv);
}

// Collision and x sweep of a node pair.  Builds the post-collision Hermite
// coefficients in the tensor-product form of the streaming sweeps, k_abc for
// a, b, c <= 2 without the fourth-order terms (index 2 pre-multiplied by
// h2(+-1) = 2/3, all pre-divided by 216, the 6^3 of the unnormalised D1Q3
// populations), from
//   A1 = j + F,  A2 = rho v v + (1 - omega) N + (1 - omega/2)(v F + F v),
//   A3 = sym(v (x) M),  M = rho v v / 3 + (1 - omega) N
// (Eq. fullstrcoll, eqts, noneqts with Guo forcing, v = u + F/(2 rho)), where
// N is the non-equilibrium second moment relative to rho v v; then streams
// them along x (warp shuffles) into X[x moment][3 c + b] (y index b, z index c).
// The forcing products come from the caller: fvaa = F_a v_a (diagonal) and
// gab = v_a F_b + F_a v_b (off-diagonal).
__device__ __forceinline__ void collide_xsweep2(float2 rho, float2 drho, float2 ux, float2 uy, float2 uz, float2 vx,
                                                float2 vy, float2 vz, float2 Fx, float2 Fy, float2 Fz, float2 nxx,
                                                float2 nyy, float2 nzz, float2 nxy, float2 nxz, float2 nyz,
                                                float2 fvxx, float2 fvyy, float2 fvzz, float2 gxy, float2 gxz,
                                                float2 gyz, float om1, float fo, float2 (&X)[3][8]) {
    const float2 rvx = rho * vx, rvy = rho * vy, rvz = rho * vz;
    const float2 exx = rvx * vx, eyy = rvy * vy, ezz = rvz * vz;
    const float2 exy = rvx * vy, exz = rvx * vz, eyz = rvy * vz;
    // q = (1 - omega) N and M = rho v v / 3 + q enter pre-divided by 24
    const float2 o24 = bc(om1 * (1.f / 24.f)), c72 = bc(1.f / 72.f), c24 = bc(1.f / 24.f);
    const float2 qxx = o24 * nxx, qyy = o24 * nyy, qzz = o24 * nzz;
    const float2 qxy = o24 * nxy, qxz = o24 * nxz, qyz = o24 * nyz;
    const float2 Mxx = mad(c72, exx, qxx), Myy = mad(c72, eyy, qyy), Mzz = mad(c72, ezz, qzz);
    const float2 Mxy = mad(c72, exy, qxy), Mxz = mad(c72, exz, qxz), Myz = mad(c72, eyz, qyz);

    // tensor-product Hermite coefficients k_abc, index 2 pre-multiplied by
    // 2/3, everything pre-divided by 216 (the 6^3 of the unnormalised sweeps):
    // k200 = A2xx / 72, k110 = A2xy / 24 with A2 = e + 24 q + (1 - omega/2) G
    const float2 f72 = bc(2.f * fo * (1.f / 72.f)), f24 = bc(fo * (1.f / 24.f)), third = bc(1.f / 3.f);
    const float2 k000 = (1.f / 216.f) * drho;
    const float2 k100 = c72 * mad(rho, ux, Fx), k010 = c72 * mad(rho, uy, Fy), k001 = c72 * mad(rho, uz, Fz);
    const float2 k200 = mad(c72, exx, mad(third, qxx, f72 * fvxx));
    const float2 k020 = mad(c72, eyy, mad(third, qyy, f72 * fvyy));
    const float2 k002 = mad(c72, ezz, mad(third, qzz, f72 * fvzz));
    const float2 k110 = mad(c24, exy, mad(f24, gxy, qxy));
    const float2 k101 = mad(c24, exz, mad(f24, gxz, qxz));
    const float2 k011 = mad(c24, eyz, mad(f24, gyz, qyz));
    const float2 tx = 2.f * vx, ty = 2.f * vy, tz = 2.f * vz;
    const float2 k210 = mad(tx, Mxy, vy * Mxx);
    const float2 k201 = mad(tx, Mxz, vz * Mxx);
    const float2 k120 = mad(ty, Mxy, vx * Myy);
    const float2 k021 = mad(ty, Myz, vz * Myy);
    const float2 k102 = mad(tz, Mxz, vx * Mzz);
    const float2 k012 = mad(tz, Myz, vy * Mzz);
    const float2 k111 = 3.f * mad(vx, Myz, mad(vy, Mxz, vz * Mxy));

    xsweep2(k000, k100, k200, X[0][0], X[1][0], X[2][0]);
    xsweep2(k010, k110, k210, X[0][1], X[1][1], X[2][1]);
    xsweep2_01(k020, k120, X[0][2], X[1][2], X[2][2]);
    xsweep2(k001, k101, k201, X[0][3], X[1][3], X[2][3]);
    xsweep2_01(k011, k111, X[0][4], X[1][4], X[2][4]);
    xsweep2_0(k021, X[0][5], X[1][5], X[2][5]);
    xsweep2_01(k002, k102, X[0][6], X[1][6], X[2][6]);
    xsweep2_0(k012, X[0][7], X[1][7], X[2][7]);
}

}  // namespace
}  // namespace tslb
