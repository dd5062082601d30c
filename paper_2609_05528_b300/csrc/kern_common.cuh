// Device helpers shared by the apply kernels (forward in apply.cu, adjoint in
// adjoint.cu): fixed-order arithmetic, arm row maps, bounded mbarrier waits,
// dependent launches and the tensor-map encoder.
#pragma once

#include <cuda.h>  // CUtensorMap and its enums (types only; no driver-library link)
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "rtt_internal.cuh"

namespace rtt {

// input row of an output row under the arm mask
__device__ __forceinline__ int seg_in_row(const ArmSeg& s, int row_out) {
    int r = row_out;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (i < s.n && r < s.len[i]) return s.begin[i] + r;
        if (i < s.n) r -= s.len[i];
    }
    return -1;
}

// output row of an input row under the arm mask, -1 if not selected
__device__ __forceinline__ int seg_out_row(const ArmSeg& s, int row_in) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (i < s.n && row_in >= s.begin[i] && row_in < s.begin[i] + s.len[i])
            return s.out_off[i] + (row_in - s.begin[i]);
    }
    return -1;
}

// Fixed-order arithmetic shared by every kernel variant, so that the variant
// (chosen from the batch size and alignment) never changes an output bit:
// fmac(a, b, c) = a b + c with one rounding.
__device__ __forceinline__ float fmac(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmac(double a, double b, double c) { return __fma_rn(a, b, c); }

// a v + (c0, c1, c2, c3) per component with packed FP32 pairs (the fused
// multiply-add of fmac on each component, two per instruction)
__device__ __forceinline__ void fmac2x2(float a, const float4& v, float& c0, float& c1, float& c2,
                                        float& c3) {
    const float2 a2 = make_float2(a, a);
    const float2 lo = __ffma2_rn(a2, make_float2(v.x, v.y), make_float2(c0, c1));
    const float2 hi = __ffma2_rn(a2, make_float2(v.z, v.w), make_float2(c2, c3));
    c0 = lo.x;
    c1 = lo.y;
    c2 = hi.x;
    c3 = hi.y;
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may be scheduled while the previous kernel in its stream is
// still finishing; it waits here, before touching any global memory, until
// that kernel has completed and its writes are visible.  Without the launch
// attribute the wait returns at once.
__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
static cudaError_t launch_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                    cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// corner weights of one ray: the FP32 table, or its BF16 copy (4 x 16 bits,
// corners 0 and 1 in .x, 2 and 3 in .y, low half first) widened exactly; the
// FP32 table then holds the same BF16-rounded values, so either read gives
// the same operand
__device__ __forceinline__ float4 corner_weights(const float4* W, const uint2* W16, int64_t e) {
    if (W16) {
        const uint2 v = W16[e];
        return make_float4(__uint_as_float(v.x << 16), __uint_as_float(v.x & 0xffff0000u),
                           __uint_as_float(v.y << 16), __uint_as_float(v.y & 0xffff0000u));
    }
    return W[e];
}

__device__ __forceinline__ int64_t floor_div(int64_t a, int64_t d) {
    return a >= 0 ? a / d : -((-a + d - 1) / d);
}

// Every mbarrier wait is bounded: on timeout the caller sets bit 0 of the
// operator's device status word, waits (bounded) for its other copies in
// flight and returns.
constexpr int kSpinLimit = 1 << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (int it = 0; it < kSpinLimit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

inline int sm_count() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

// one wave of resident CTAs of `kernel` for a persistent loop (fewer when the
// work needs fewer)
template <typename Kern>
static int resident_grid(Kern kernel, int threads, size_t smem, int64_t n_tasks, int warps) {
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const int64_t want = (n_tasks + warps - 1) / warps;
    const int64_t cap = (int64_t)sm_count() * per_sm;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); null when unavailable
inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

// frames per hat step when that is an integer the periodic kernels handle
// (2, 4 or 8), else 0
inline int frames_per_hat(int64_t D) {
    if (D <= 0 || kFracOne % D != 0) return 0;
    const int P = (int)(kFracOne / D);
    return (P == 2 || P == 4 || P == 8) ? P : 0;
}

}  // namespace rtt
