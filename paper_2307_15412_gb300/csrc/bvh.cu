// bvh.cu -- linear BVH builder for the per-frame triangle mesh.
//
// The paper's scene is a triangle mesh that is re-posed every frame
// (Sec. III), so the acceleration structure is rebuilt per frame:
//   1. k_tri_prep   per triangle: bounding-box centre, per-block centre
//                   bounds, reset of the bottom-up visit flags
//   2. k_sort       one CTA: scene centre bounds, 30-bit Morton codes,
//                   stable LSD radix sort (4 x 8-bit digits) of (code, id)
//   3. k_hierarchy  per leaf: gather the triangle in Morton order, then
//                   climb the binary radix tree (Karras, HPG 2012) bottom
//                   up, deciding each parent from the neighbouring key
//                   differences (Apetrei, EG 2014) and merging child boxes
//                   on the way (the second thread to reach a node goes on).
// Internal node ids are split positions gamma in [0, n-2]; leaves are
// ~position.  Keys are made distinct by appending the sorted position.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rr_internal.cuh"

namespace rr {
namespace {

constexpr int kPrepThreads = 256;
constexpr int kSortThreads = 1024;
constexpr int kSortItems = 8;                         // keys per lane per slice
constexpr int kSlice = kSortThreads * kSortItems;     // keys per slice
constexpr int kCntStride = 33;                        // padded [digit][warp] counters

__device__ __forceinline__ uint32_t spread10(uint32_t v) {
  v &= 0x3FFu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

__global__ void __launch_bounds__(kPrepThreads)
k_tri_prep(const float *__restrict__ V, const int32_t *__restrict__ F, int n,
           float4 *__restrict__ cent, float *__restrict__ blockbounds, int32_t *__restrict__ flags) {
  const int i = blockIdx.x * kPrepThreads + threadIdx.x;
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  if (i < n) {
    const int a = F[3 * i], b = F[3 * i + 1], c = F[3 * i + 2];
    float cc[3];
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      const float va = V[3 * a + x], vb = V[3 * b + x], vc = V[3 * c + x];
      const float mn = fminf(va, fminf(vb, vc)), mx = fmaxf(va, fmaxf(vb, vc));
      cc[x] = __fmul_rn(__fadd_rn(mn, mx), 0.5f);  // same rounding as the integer-step definition
      lo[x] = hi[x] = cc[x];
    }
    cent[i] = make_float4(cc[0], cc[1], cc[2], 0.f);
    flags[i] = -1;
  }
  // block reduction of the centre bounds
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[x] = fminf(lo[x], __shfl_xor_sync(0xffffffffu, lo[x], o));
      hi[x] = fmaxf(hi[x], __shfl_xor_sync(0xffffffffu, hi[x], o));
    }
  }
  __shared__ float red[kPrepThreads / 32][6];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
#pragma unroll
    for (int x = 0; x < 3; ++x) { red[w][x] = lo[x]; red[w][3 + x] = hi[x]; }
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    const int x = threadIdx.x;
    float v = red[0][x];
    for (int k = 1; k < kPrepThreads / 32; ++k) v = x < 3 ? fminf(v, red[k][x]) : fmaxf(v, red[k][x]);
    blockbounds[6 * blockIdx.x + x] = v;
  }
}

__global__ void __launch_bounds__(kSortThreads, 1)
k_sort(int n, int nblk, const float *__restrict__ blockbounds, const float4 *__restrict__ cent,
       uint32_t *keys, uint32_t *keys_alt, int32_t *ids, int32_t *ids_alt, BvhHeader *hdr) {
  __shared__ float s_lo[3], s_hi[3];
  __shared__ uint32_t s_hist[4][256];
  __shared__ uint32_t s_run[256];
  __shared__ uint32_t s_cnt[256 * kCntStride];
  __shared__ uint32_t s_wsum[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // 1. scene centre bounds
  if (tid < 6) {
    float v = tid < 3 ? INFINITY : -INFINITY;
    for (int b = 0; b < nblk; ++b) v = tid < 3 ? fminf(v, blockbounds[6 * b + tid]) : fmaxf(v, blockbounds[6 * b + tid]);
    if (tid < 3) s_lo[tid] = v; else s_hi[tid - 3] = v;
  }
  for (int x = tid; x < 4 * 256; x += kSortThreads) (&s_hist[0][0])[x] = 0;
  __syncthreads();

  // 2. Morton codes and the four digit histograms
  float ext[3], lo[3];
#pragma unroll
  for (int x = 0; x < 3; ++x) { lo[x] = s_lo[x]; ext[x] = __fsub_rn(s_hi[x], s_lo[x]); }
  for (int i = tid; i < n; i += kSortThreads) {
    const float4 c = cent[i];
    const float cc[3] = {c.x, c.y, c.z};
    uint32_t q[3];
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      if (ext[x] > 0.f) {
        float u = __fdiv_rn(__fsub_rn(cc[x], lo[x]), ext[x]);
        u = __fmul_rn(u, 1024.f);
        int qi = (int)floorf(u);
        q[x] = (uint32_t)min(max(qi, 0), 1023);
      } else {
        q[x] = 0u;
      }
    }
    const uint32_t code = (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
    keys[i] = code;
    ids[i] = i;
#pragma unroll
    for (int p = 0; p < 4; ++p) atomicAdd(&s_hist[p][(code >> (8 * p)) & 255u], 1u);
  }
  __syncthreads();
  // exclusive scans of the histograms (one warp per pass)
  if (warp < 4) {
    uint32_t carry = 0;
    for (int base = 0; base < 256; base += 32) {
      uint32_t v = s_hist[warp][base + lane], incl = v;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      s_hist[warp][base + lane] = carry + incl - v;
      carry += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
  __syncthreads();

  // 3. four stable scatter passes
  const uint32_t lt_mask = (1u << lane) - 1u;
  for (int p = 0; p < 4; ++p) {
    const uint32_t *src_k = (p & 1) ? keys_alt : keys;
    const int32_t *src_i = (p & 1) ? ids_alt : ids;
    uint32_t *dst_k = (p & 1) ? keys : keys_alt;
    int32_t *dst_i = (p & 1) ? ids : ids_alt;
    const int shift = 8 * p;
    if (tid < 256) s_run[tid] = s_hist[p][tid];
    for (int base = 0; base < n; base += kSlice) {
      for (int x = tid; x < 256 * kCntStride; x += kSortThreads) s_cnt[x] = 0;
      __syncthreads();
      uint32_t k[kSortItems];
      int32_t id[kSortItems];
      uint32_t rank[kSortItems];
#pragma unroll
      for (int j = 0; j < kSortItems; ++j) {
        const int idx = base + (warp * kSortItems + j) * 32 + lane;
        const bool ok = idx < n;
        k[j] = ok ? src_k[idx] : 0u;
        id[j] = ok ? src_i[idx] : 0;
        const uint32_t dg = ok ? ((k[j] >> shift) & 255u) : 256u + lane;
        const uint32_t peers = __match_any_sync(0xffffffffu, dg);
        uint32_t before = 0;
        if (ok) before = s_cnt[dg * kCntStride + warp];
        __syncwarp();
        if (ok && (peers & lt_mask) == 0u) s_cnt[dg * kCntStride + warp] = before + __popc(peers);
        __syncwarp();
        rank[j] = before + __popc(peers & lt_mask);
      }
      __syncthreads();
      // exclusive scan of the counters in (digit, warp) order: thread t owns
      // digit t/4 and warps 8*(t%4) .. 8*(t%4)+7
      {
        const int dg = tid >> 2, w0 = (tid & 3) * 8;
        uint32_t v[8], s = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) { v[q] = s_cnt[dg * kCntStride + w0 + q]; s += v[q]; }
        uint32_t incl = s;
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += t;
        }
        if (lane == 31) s_wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
          const uint32_t x = s_wsum[lane];
          uint32_t xi = x;
          for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += t;
          }
          s_wsum[lane] = xi - x;
        }
        __syncthreads();
        uint32_t run = s_wsum[warp] + incl - s;
#pragma unroll
        for (int q = 0; q < 8; ++q) { s_cnt[dg * kCntStride + w0 + q] = run; run += v[q]; }
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < kSortItems; ++j) {
        const int idx = base + (warp * kSortItems + j) * 32 + lane;
        if (idx < n) {
          const uint32_t dg = (k[j] >> shift) & 255u;
          const uint32_t dest = s_run[dg] + (s_cnt[dg * kCntStride + warp] - s_cnt[dg * kCntStride]) + rank[j];
          dst_k[dest] = k[j];
          dst_i[dest] = id[j];
        }
      }
      __syncthreads();
      if (tid < 256) {
        const int slice_n = min(kSlice, n - base);
        const uint32_t next = tid < 255 ? s_cnt[(tid + 1) * kCntStride] : (uint32_t)slice_n;
        s_run[tid] += next - s_cnt[tid * kCntStride];
      }
      __syncthreads();
    }
  }
  if (tid == 0) hdr->n = n;
}

__device__ __forceinline__ uint64_t key_delta(const uint32_t *keys, int x) {
  // XOR of the augmented keys (code << 32 | position) at x and x + 1
  return ((uint64_t)(keys[x] ^ keys[x + 1]) << 32) | (uint32_t)(x ^ (x + 1));
}

// Leaf i of the bottom-up climb (Apetrei 2014 order over the sorted keys):
// writes the leaf's triangle in Morton order and its box into the parent,
// and the second of two siblings to arrive goes on with their union; the
// root's thread writes the header.  The flags must be -1 on entry.
__device__ __forceinline__ void climb_leaf(int i, int n, const uint32_t *__restrict__ keys, const int32_t *__restrict__ ids,
                                           const float *__restrict__ V, const int32_t *__restrict__ F, BvhNode *nodes,
                                           float4 *__restrict__ tris, int32_t *flags, BvhHeader *hdr) {
  const int tid = ids[i];
  const int a = F[3 * tid], b = F[3 * tid + 1], c = F[3 * tid + 2];
  const float3 v0 = make_float3(V[3 * a], V[3 * a + 1], V[3 * a + 2]);
  const float3 v1 = make_float3(V[3 * b], V[3 * b + 1], V[3 * b + 2]);
  const float3 v2 = make_float3(V[3 * c], V[3 * c + 1], V[3 * c + 2]);
  tris[3 * i + 0] = make_float4(v0.x, v0.y, v0.z, __int_as_float(tid));
  tris[3 * i + 1] = make_float4(v1.x, v1.y, v1.z, 0.f);
  tris[3 * i + 2] = make_float4(v2.x, v2.y, v2.z, 0.f);
  float3 lo = make_float3(fminf(v0.x, fminf(v1.x, v2.x)), fminf(v0.y, fminf(v1.y, v2.y)), fminf(v0.z, fminf(v1.z, v2.z)));
  float3 hi = make_float3(fmaxf(v0.x, fmaxf(v1.x, v2.x)), fmaxf(v0.y, fmaxf(v1.y, v2.y)), fmaxf(v0.z, fmaxf(v1.z, v2.z)));
  if (n == 1) {
    hdr->root = ~0;
    hdr->lo[0] = lo.x; hdr->lo[1] = lo.y; hdr->lo[2] = lo.z;
    hdr->hi[0] = hi.x; hdr->hi[1] = hi.y; hdr->hi[2] = hi.z;
    return;
  }
  int cur = ~i, l = i, r = i;
  for (int guard = 0; guard < 2 * n + 64; ++guard) {
    bool as_left;
    if (l == 0) as_left = true;
    else if (r == n - 1) as_left = false;
    else as_left = key_delta(keys, r) < key_delta(keys, l - 1);
    const int p = as_left ? r : l - 1;
    BvhNode *np = nodes + p;
    if (as_left) {
      np->lxy = make_float4(lo.x, hi.x, lo.y, hi.y);
      reinterpret_cast<float2 *>(&np->lrz)[0] = make_float2(lo.z, hi.z);
      np->kids.x = cur;
    } else {
      np->rxy = make_float4(lo.x, hi.x, lo.y, hi.y);
      reinterpret_cast<float2 *>(&np->lrz)[1] = make_float2(lo.z, hi.z);
      np->kids.y = cur;
    }
    // release: this child's box is visible before the flag; acquire: the
    // sibling's box is visible after it (no full fences on the climb)
    int other;
    asm volatile("atom.acq_rel.gpu.global.exch.b32 %0, [%1], %2;"
                 : "=r"(other)
                 : "l"(flags + p), "r"(as_left ? l : r)
                 : "memory");
    if (other < 0) return;  // first to arrive: the sibling's thread goes on
    float4 sxy;
    float2 sz;
    if (as_left) {
      sxy = __ldcg(&np->rxy);
      sz = __ldcg(reinterpret_cast<const float2 *>(&np->lrz) + 1);
      r = other;
    } else {
      sxy = __ldcg(&np->lxy);
      sz = __ldcg(reinterpret_cast<const float2 *>(&np->lrz));
      l = other;
    }
    lo = make_float3(fminf(lo.x, sxy.x), fminf(lo.y, sxy.z), fminf(lo.z, sz.x));
    hi = make_float3(fmaxf(hi.x, sxy.y), fmaxf(hi.y, sxy.w), fmaxf(hi.z, sz.y));
    cur = p;
    if (l == 0 && r == n - 1) {
      hdr->root = p;
      hdr->lo[0] = lo.x; hdr->lo[1] = lo.y; hdr->lo[2] = lo.z;
      hdr->hi[0] = hi.x; hdr->hi[1] = hi.y; hdr->hi[2] = hi.z;
      return;
    }
  }
}


__global__ void __launch_bounds__(kPrepThreads)
k_hierarchy(int n, const uint32_t *__restrict__ keys, const int32_t *__restrict__ ids,
            const float *__restrict__ V, const int32_t *__restrict__ F, BvhNode *nodes,
            float4 *__restrict__ tris, int32_t *flags, BvhHeader *hdr) {
  const int i = blockIdx.x * kPrepThreads + threadIdx.x;
  if (i >= n) return;
  climb_leaf(i, n, keys, ids, V, F, nodes, tris, flags, hdr);
}

// The refit job of block b (jobs[j].blk0 <= b < jobs[j + 1].blk0).
__device__ __forceinline__ int refit_job_of(const BuildJob *jobs, int n_jobs, int b) {
  int lo = 0, hi = n_jobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].blk0 <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(kRefitThreads) k_refit_reset(const BuildJob *__restrict__ jobs, int n_jobs) {
  const BuildJob &J = jobs[refit_job_of(jobs, n_jobs, blockIdx.x)];
  const int i = ((int)blockIdx.x - J.blk0) * kRefitThreads + threadIdx.x;
  if (i < J.n) J.flags[i] = -1;
}

__global__ void __launch_bounds__(kRefitThreads) k_refit(const BuildJob *__restrict__ jobs, int n_jobs) {
  const BuildJob &J = jobs[refit_job_of(jobs, n_jobs, blockIdx.x)];
  const int i = ((int)blockIdx.x - J.blk0) * kRefitThreads + threadIdx.x;
  if (i < J.n) climb_leaf(i, J.n, J.keys, J.ids, J.V, J.F, J.nodes, J.tris, J.flags, J.hdr);
}

__global__ void k_empty_header(BvhHeader *hdr) {
  hdr->n = 0;
  hdr->root = 0;
  for (int x = 0; x < 3; ++x) { hdr->lo[x] = INFINITY; hdr->hi[x] = -INFINITY; }
}

}  // namespace

cudaError_t launch_refit_bvh(SceneDev &s, cudaStream_t st) {
  const int n = (int)s.nt;
  if (n == 0) {
    k_empty_header<<<1, 1, 0, st>>>(s.hdr);
    return cudaGetLastError();
  }
  cudaError_t e = cudaMemsetAsync(s.flags, 0xff, sizeof(int32_t) * (size_t)n, st);
  if (e != cudaSuccess) return e;
  k_hierarchy<<<(n + kPrepThreads - 1) / kPrepThreads, kPrepThreads, 0, st>>>(n, s.keys, s.ids, s.V, s.F, s.nodes,
                                                                              s.tris, s.flags, s.hdr);
  return cudaGetLastError();
}

cudaError_t launch_refit_batch(const BuildJob *jobs, int n_jobs, int blocks, cudaStream_t st) {
  if (n_jobs < 1 || blocks < 1) return cudaSuccess;
  k_refit_reset<<<blocks, kRefitThreads, 0, st>>>(jobs, n_jobs);
  k_refit<<<blocks, kRefitThreads, 0, st>>>(jobs, n_jobs);
  return cudaGetLastError();
}

cudaError_t launch_build_bvh(SceneDev &s, cudaStream_t st) {
  const int n = (int)s.nt;
  bool used = false;
  cudaError_t ce = launch_build_bvh_cluster(s, st, &used);
  if (ce != cudaSuccess || used) return ce;
  if (n == 0) {
    k_empty_header<<<1, 1, 0, st>>>(s.hdr);
    return cudaGetLastError();
  }
  const int nblk = (n + kPrepThreads - 1) / kPrepThreads;
  k_tri_prep<<<nblk, kPrepThreads, 0, st>>>(s.V, s.F, n, s.cent, s.blockbounds, s.flags);
  k_sort<<<1, kSortThreads, 0, st>>>(n, nblk, s.blockbounds, s.cent, s.keys, s.keys_alt, s.ids, s.ids_alt, s.hdr);
  k_hierarchy<<<nblk, kPrepThreads, 0, st>>>(n, s.keys, s.ids, s.V, s.F, s.nodes, s.tris, s.flags, s.hdr);
  return cudaGetLastError();
}

}  // namespace rr
