// Fused deterministic adjoint A^T (Sec. 5: explicit adjoint action) for the
// FP32 path, without the per-ray scratch round trip.
//
// The source nodes are cut into tiles of kTR x kTP nodes.  At build time
// every ray is listed once per tile that holds one of its four bilinear
// corners ("visits", sorted by (tile, ray), with a 4-bit corner mask).  One
// CTA takes a chunk of a tile's visits: for each visit it stages the ray's
// data row y[row][0..T)[b0..b0+BC) in shared memory with cp.async (3-stage
// ring), contracts it over frames into z[k][b] = sum_f h(f, k) y[f][b] with
// the exact fixed-point hat arithmetic of the forward, and adds W_c z into
// the shared accumulators of the corners that lie in the tile.  Each
// accumulator slot (node, k, b) is updated by one thread in visit order, so
// the result is deterministic without atomics.  Tiles whose visit list is
// split over several CTAs write partial tiles that a second kernel adds in
// chunk order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cub/cub.cuh>
#include <vector>

#include "rtt_internal.cuh"

namespace rtt {

constexpr int kTR = 2;                 // tile height (radial nodes)
constexpr int kTP = 8;                 // tile width (azimuthal nodes)
constexpr int kTN = kTR * kTP;         // nodes per tile
constexpr int kFusedThreads = 256;
constexpr int kStages = 3;
constexpr int kChunkVisits = 256;      // visits per CTA before a tile is split
constexpr uint32_t kVisitRayMask = (1u << 28) - 1;

__device__ __forceinline__ int64_t fdiv_floor(int64_t a, int64_t d) {
    return a >= 0 ? a / d : -((-a + d - 1) / d);
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

struct FusedArgs {
    const int32_t* ray_row;
    const int32_t* node00;
    const int32_t* node01;
    const float4* W;
    const int32_t* K0;
    const int32_t* F0;
    const uint32_t* visits;  // e | mask << 28
    const int4* items;       // (tile, v_begin, v_end, partial slot or -1)
    const float* y;          // offset to the batch chunk
    float* x;                // offset to the batch chunk
    float* partial;          // [slots][kTN][K][BC]
    ArmSeg seg;
    int B, K, Tn, n_r, n_phi, n_tp;
    int64_t D;
};

__device__ __forceinline__ int seg_out(const ArmSeg& s, int row_in) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
        if (i < s.n && row_in >= s.begin[i] && row_in < s.begin[i] + s.len[i])
            return s.out_off[i] + (row_in - s.begin[i]);
    return -1;
}

// local index of node (i, j) in the tile whose first node is (ib, jb), or -1
__device__ __forceinline__ int local_of(int node, int n_phi, int ib, int jb) {
    const int i = node / n_phi, j = node - i * n_phi;
    const int di = i - ib, dj = j - jb;
    return (di >= 0 && di < kTR && dj >= 0 && dj < kTP) ? di * kTP + dj : -1;
}

template <int BC>
__global__ void __launch_bounds__(kFusedThreads) adj_fused_kernel(const FusedArgs f) {
    extern __shared__ __align__(16) float fsm[];
    constexpr int Q = BC / 4;
    float* acc = fsm;                          // [kTN][K][BC]
    float* ybuf = acc + kTN * f.K * BC;        // [kStages][Tn][BC]
    const int tid = threadIdx.x;
    const int4 item = f.items[blockIdx.x];
    const int tile = item.x, v0 = item.y, v1 = item.z, slot = item.w;
    const int ti = tile / f.n_tp, tp = tile - ti * f.n_tp;
    const int i_base = ti * kTR, j_base = tp * kTP;
    for (int o = tid; o < kTN * f.K * BC; o += kFusedThreads) acc[o] = 0.0f;
    const int row_chunks = f.Tn * Q;  // 16-byte chunks per staged row
    // copy visit v's data row into stage s (nothing if the ray is outside the arm)
    auto stage_in = [&](int v, int s) {
        if (v < v1) {
            const int e = (int)(f.visits[v] & kVisitRayMask);
            const int row_out = seg_out(f.seg, f.ray_row[e]);
            if (row_out >= 0) {
                const float* src = f.y + (int64_t)row_out * f.Tn * f.B;
                float* dst = ybuf + (int64_t)s * f.Tn * BC;
                for (int o = tid; o < row_chunks; o += kFusedThreads) {
                    const int fr = o / Q, q = o - fr * Q;
                    cp_async16(dst + fr * BC + 4 * q, src + (int64_t)fr * f.B + 4 * q);
                }
            }
        }
        cp_async_commit();
    };
#pragma unroll
    for (int s = 0; s < kStages - 1; ++s) stage_in(v0 + s, s);
    const int n_items_k = f.K * Q;  // (hat, batch quad) work items
    for (int v = v0; v < v1; ++v) {
        stage_in(v + kStages - 1, (v - v0 + kStages - 1) % kStages);
        cp_async_wait<kStages - 1>();
        __syncthreads();
        const uint32_t code = f.visits[v];
        const int e = (int)(code & kVisitRayMask);
        const int row_out = seg_out(f.seg, f.ray_row[e]);
        if (row_out >= 0) {
            const float* ys = ybuf + (int64_t)((v - v0) % kStages) * f.Tn * BC;
            const float4 wv = f.W[e];
            const int n00 = f.node00[e], n01 = f.node01[e];
            const int loc0 = local_of(n00, f.n_phi, i_base, j_base);
            const int loc1 = local_of(n00 + f.n_phi, f.n_phi, i_base, j_base);
            const int loc2 = local_of(n01, f.n_phi, i_base, j_base);
            const int loc3 = local_of(n01 + f.n_phi, f.n_phi, i_base, j_base);
            const int64_t U0 = (int64_t)f.K0[e] * kFracOne + (int64_t)f.F0[e];
            for (int it = tid; it < n_items_k; it += kFusedThreads) {
                const int k = it / Q, q = it - k * Q;
                float4 s4 = make_float4(0.f, 0.f, 0.f, 0.f);
                const int64_t hi_excl = (int64_t)(k + 1) * kFracOne;
                const int64_t lo_incl = (int64_t)(k - 1) * kFracOne;
                const float est = (float)(U0 - hi_excl) * (1.0f / (float)f.D);
                int fr = (int)fminf(fmaxf(floorf(est) - 1.0f, 0.0f), (float)f.Tn);
                int64_t U = U0 - (int64_t)fr * f.D;
                while (fr < f.Tn && U >= hi_excl) { ++fr; U -= f.D; }
                for (; fr < f.Tn && U >= lo_incl; ++fr, U -= f.D) {
                    const int k0 = (int)(U >> kFracBits);
                    const float fq = (float)(int32_t)(U & kFracMask) * (1.0f / (float)kFracOne);
                    const float hw = (k0 == k) ? 1.0f - fq : fq;
                    const float4 t = reinterpret_cast<const float4*>(ys + fr * BC)[q];
                    s4.x += hw * t.x;
                    s4.y += hw * t.y;
                    s4.z += hw * t.z;
                    s4.w += hw * t.w;
                }
                // scatter into the tile's accumulators: slot (node, k, quad) is
                // owned by this thread, updated in visit order
                const int kq = (k * BC) + 4 * q;
                if (loc0 >= 0) {
                    float4* a4 = reinterpret_cast<float4*>(acc + loc0 * f.K * BC + kq);
                    float4 t = *a4;
                    t.x += wv.x * s4.x; t.y += wv.x * s4.y; t.z += wv.x * s4.z; t.w += wv.x * s4.w;
                    *a4 = t;
                }
                if (loc1 >= 0) {
                    float4* a4 = reinterpret_cast<float4*>(acc + loc1 * f.K * BC + kq);
                    float4 t = *a4;
                    t.x += wv.y * s4.x; t.y += wv.y * s4.y; t.z += wv.y * s4.z; t.w += wv.y * s4.w;
                    *a4 = t;
                }
                if (loc2 >= 0) {
                    float4* a4 = reinterpret_cast<float4*>(acc + loc2 * f.K * BC + kq);
                    float4 t = *a4;
                    t.x += wv.z * s4.x; t.y += wv.z * s4.y; t.z += wv.z * s4.z; t.w += wv.z * s4.w;
                    *a4 = t;
                }
                if (loc3 >= 0) {
                    float4* a4 = reinterpret_cast<float4*>(acc + loc3 * f.K * BC + kq);
                    float4 t = *a4;
                    t.x += wv.w * s4.x; t.y += wv.w * s4.y; t.z += wv.w * s4.z; t.w += wv.w * s4.w;
                    *a4 = t;
                }
            }
        }
        __syncthreads();  // the stage of visit v is refilled two iterations later
    }
    cp_async_wait<0>();
    __syncthreads();
    // write the tile: final x when the tile is one chunk, else a partial tile
    for (int o = tid; o < kTN * f.K * Q; o += kFusedThreads) {
        const int l = o / (f.K * Q);
        const int rem = o - l * (f.K * Q);
        const int k = rem / Q, q = rem - k * Q;
        const float4 val = reinterpret_cast<const float4*>(acc + l * f.K * BC + k * BC)[q];
        if (slot >= 0) {
            reinterpret_cast<float4*>(f.partial + ((int64_t)slot * kTN + l) * f.K * BC + k * BC)[q] = val;
        } else {
            const int i = i_base + l / kTP, j = j_base + (l % kTP);
            if (i < f.n_r && j < f.n_phi) {
                const int node = i * f.n_phi + j;
                reinterpret_cast<float4*>(f.x + ((int64_t)node * f.K + k) * f.B)[q] = val;
            }
        }
    }
}

// x of a split tile = sum of its partial tiles in chunk order
__global__ void adj_fused_reduce(const int4* split_tiles, int n_split, const float* partial, int K,
                                 int BC, int B, int n_r, int n_phi, int n_tp, float* x) {
    const int st = blockIdx.x;
    if (st >= n_split) return;
    const int4 t = split_tiles[st];  // (tile, first slot, n_slots, -)
    const int ti = t.x / n_tp, tp = t.x - ti * n_tp;
    for (int o = threadIdx.x; o < kTN * K * BC; o += blockDim.x) {
        float s = 0.0f;
        for (int c = 0; c < t.z; ++c) s += partial[(int64_t)(t.y + c) * kTN * K * BC + o];
        const int l = o / (K * BC), rem = o - l * K * BC;
        const int k = rem / BC, b = rem - k * BC;
        const int i = ti * kTR + l / kTP, j = tp * kTP + (l % kTP);
        if (i < n_r && j < n_phi) x[((int64_t)(i * n_phi + j) * K + k) * B + b] = s;
    }
}

// ---------------------------------------------------------------------------
// Build-time visit lists: every (tile, ray) pair with the corners it holds.
// ---------------------------------------------------------------------------
__global__ void visit_keys(int64_t E, int n_phi, int n_tp, const int32_t* node00,
                           const int32_t* node01, unsigned long long* key, int32_t* val) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 4 * E) return;
    const int64_t e = t >> 2;
    const int c = (int)(t & 3);
    const int node = (c == 0) ? node00[e] : (c == 1) ? node00[e] + n_phi
                   : (c == 2) ? node01[e] : node01[e] + n_phi;
    const int i = node / n_phi, j = node - i * n_phi;
    const int tile = (i / kTR) * n_tp + j / kTP;
    key[t] = ((unsigned long long)tile << 32) | (unsigned long long)e;
    val[t] = c;
}

__global__ void visit_heads(int64_t n, const unsigned long long* key, const int32_t* val,
                            int32_t* head, uint32_t* code, unsigned int* tile_count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bool h = (i == 0) || key[i] != key[i - 1];
    head[i] = h ? 1 : 0;
    if (h) {
        int mask = 0;
        for (int64_t j = i; j < n && j < i + 4 && key[j] == key[i]; ++j) mask |= 1 << val[j];
        code[i] = (uint32_t)(key[i] & 0xffffffffull) | ((uint32_t)mask << 28);
        atomicAdd(&tile_count[key[i] >> 32], 1u);  // integer count: order independent
    }
}

__global__ void visit_compact(int64_t n, const int32_t* head, const int32_t* pos,
                              const uint32_t* code, uint32_t* visits) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !head[i]) return;
    visits[pos[i]] = code[i];
}

}  // namespace rtt

using namespace rtt;

namespace rtt {

// Builds op->visits, op->tile_ptr and the work items; host part is small.
rtt_status build_visits(rtt_op_s* op, cudaStream_t st) {
    const int64_t E = op->n_rays;
    if (E >= (int64_t)kVisitRayMask) return RTT_OK;  // too many rays: two-phase adjoint only
    const int n_phi = op->grid.n_phi, n_r = op->grid.n_r;
    const int n_tr = (n_r + kTR - 1) / kTR, n_tp = (n_phi + kTP - 1) / kTP;
    const int n_tiles = n_tr * n_tp;
    const int64_t n = 4 * E;
    unsigned long long *k_in = nullptr, *k_out = nullptr;
    int32_t *v_in = nullptr, *v_out = nullptr, *head = nullptr, *pos = nullptr;
    uint32_t* code = nullptr;
    unsigned int* cnt = nullptr;
    void* tmp = nullptr;
    size_t tb1 = 0, tb2 = 0, tb3 = 0;
    int end_bit = 32;
    while ((1ll << (end_bit - 32)) < n_tiles) ++end_bit;
    cub::DeviceRadixSort::SortPairs(nullptr, tb1, k_in, k_out, v_in, v_out, n, 0, end_bit, st);
    cub::DeviceScan::ExclusiveSum(nullptr, tb2, head, pos, n, st);
    cub::DeviceScan::ExclusiveSum(nullptr, tb3, cnt, cnt, n_tiles + 1, st);
    size_t tb = tb1 > tb2 ? tb1 : tb2;
    tb = tb > tb3 ? tb : tb3;
    cudaError_t e = cudaMalloc(&k_in, n * 8);
    if (e == cudaSuccess) e = cudaMalloc(&k_out, n * 8);
    if (e == cudaSuccess) e = cudaMalloc(&v_in, n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&v_out, n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&head, n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&pos, n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&code, n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&cnt, (n_tiles + 1) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&tmp, tb + 16);
    int32_t n_vis = 0, last_head = 0;
    std::vector<unsigned int> tile_ptr(n_tiles + 1);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, (n_tiles + 1) * 4, st);
    if (e == cudaSuccess) {
        visit_keys<<<(int)((n + 255) / 256), 256, 0, st>>>(E, n_phi, n_tp, op->node00, op->node01,
                                                            k_in, v_in);
        e = cudaGetLastError();
    }
    size_t t1 = tb;
    if (e == cudaSuccess)
        e = cub::DeviceRadixSort::SortPairs(tmp, t1, k_in, k_out, v_in, v_out, n, 0, end_bit, st);
    if (e == cudaSuccess) {
        visit_heads<<<(int)((n + 255) / 256), 256, 0, st>>>(n, k_out, v_out, head, code, cnt);
        e = cudaGetLastError();
    }
    t1 = tb;
    if (e == cudaSuccess) e = cub::DeviceScan::ExclusiveSum(tmp, t1, head, pos, n, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&n_vis, pos + (n - 1), 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&last_head, head + (n - 1), 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    n_vis += last_head;
    if (e == cudaSuccess) e = cudaMalloc(&op->visits, (size_t)n_vis * 4 + 16);
    if (e == cudaSuccess) {
        visit_compact<<<(int)((n + 255) / 256), 256, 0, st>>>(n, head, pos, code, op->visits);
        e = cudaGetLastError();
    }
    t1 = tb;
    if (e == cudaSuccess) e = cub::DeviceScan::ExclusiveSum(tmp, t1, cnt, cnt, n_tiles + 1, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(tile_ptr.data(), cnt, (n_tiles + 1) * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(k_in);
    cudaFree(k_out);
    cudaFree(v_in);
    cudaFree(v_out);
    cudaFree(head);
    cudaFree(pos);
    cudaFree(code);
    cudaFree(cnt);
    cudaFree(tmp);
    if (e != cudaSuccess) {
        set_error("visit lists: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? RTT_ENOMEM : RTT_ECUDA;
    }
    // work items: (tile, v_begin, v_end, slot); split tiles get partial slots
    std::vector<int4> items, splits;
    int slots = 0;
    for (int t = 0; t < n_tiles; ++t) {
        const int b = (int)tile_ptr[t], en = (int)tile_ptr[t + 1];
        const int nv = en - b;
        const int nch = nv <= kChunkVisits ? 1 : (nv + kChunkVisits - 1) / kChunkVisits;
        if (nch == 1) {
            items.push_back(make_int4(t, b, en, -1));
        } else {
            splits.push_back(make_int4(t, slots, nch, 0));
            for (int c = 0; c < nch; ++c) {
                const int cb = b + (int)((int64_t)nv * c / nch);
                const int ce = b + (int)((int64_t)nv * (c + 1) / nch);
                items.push_back(make_int4(t, cb, ce, slots + c));
            }
            slots += nch;
        }
    }
    // heaviest items first so the tail of the grid is short
    std::stable_sort(items.begin(), items.end(),
                     [](const int4& a, const int4& b) { return (a.z - a.y) > (b.z - b.y); });
    e = cudaMalloc(&op->items, items.size() * sizeof(int4) + 16);
    if (e == cudaSuccess && !splits.empty()) e = cudaMalloc(&op->split_tiles, splits.size() * sizeof(int4) + 16);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(op->items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !splits.empty())
        e = cudaMemcpyAsync(op->split_tiles, splits.data(), splits.size() * sizeof(int4),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        set_error("visit items: %s", cudaGetErrorString(e));
        return RTT_ECUDA;
    }
    op->n_items = (int)items.size();
    op->n_split = (int)splits.size();
    op->n_partial_slots = slots;
    op->n_tp = n_tp;
    op->n_visits = n_vis;
    return RTT_OK;
}

size_t fused_partial_bytes(const rtt_op_s* op) {
    return (size_t)op->n_partial_slots * kTN * op->time.n_hats * 32 * sizeof(float);
}

// Launches the fused adjoint for one batch chunk; returns cudaErrorNotSupported
// when this configuration must use the two-phase path.
cudaError_t launch_adjoint_fused(const rtt_op_s* op, const float* y, float* x, int B, int b_first,
                                 int Bc, const ArmSeg& seg, float* partial, cudaStream_t st) {
    if (!op->items || (B % 4) != 0 || (Bc % 4) != 0) return cudaErrorNotSupported;
    const int K = op->time.n_hats, Tn = op->time.n_frames;
    int BC = Bc <= 4 ? 4 : Bc <= 8 ? 8 : Bc <= 16 ? 16 : 32;
    if (BC != Bc) return cudaErrorNotSupported;
    const size_t smem = ((size_t)kTN * K * BC + (size_t)kStages * Tn * BC) * sizeof(float);
    if (smem > 200 * 1024) return cudaErrorNotSupported;
    FusedArgs f{};
    f.ray_row = op->ray_row;
    f.node00 = op->node00;
    f.node01 = op->node01;
    f.W = op->W;
    f.K0 = op->K0;
    f.F0 = op->F0;
    f.visits = op->visits;
    f.items = (const int4*)op->items;
    f.y = y + b_first;
    f.x = x + b_first;
    f.partial = partial;
    f.seg = seg;
    f.B = B;
    f.K = K;
    f.Tn = Tn;
    f.n_r = op->grid.n_r;
    f.n_phi = op->grid.n_phi;
    f.n_tp = op->n_tp;
    f.D = op->frame_D;
    cudaError_t e = cudaSuccess;
#define RTT_FUSED_CASE(bc)                                                                    \
    case bc:                                                                                  \
        e = cudaFuncSetAttribute(adj_fused_kernel<bc>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 (int)smem);                                                  \
        if (e == cudaSuccess) adj_fused_kernel<bc><<<op->n_items, kFusedThreads, smem, st>>>(f); \
        break;
    switch (BC) {
        RTT_FUSED_CASE(4)
        RTT_FUSED_CASE(8)
        RTT_FUSED_CASE(16)
        RTT_FUSED_CASE(32)
        default: return cudaErrorNotSupported;
    }
#undef RTT_FUSED_CASE
    if (e != cudaSuccess) return e;
    e = cudaGetLastError();
    if (e != cudaSuccess || op->n_split == 0) return e;
    adj_fused_reduce<<<op->n_split, 256, 0, st>>>((const int4*)op->split_tiles, op->n_split, partial,
                                                  K, BC, B, op->grid.n_r, op->grid.n_phi, op->n_tp,
                                                  x + b_first);
    return cudaGetLastError();
}

}  // namespace rtt
