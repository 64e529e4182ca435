// trace_tris.cu -- rays cast to each mesh triangle (Sec. III: multiple rays
// are cast to each mesh triangle and the scattering of each face is
// simulated), and the alpha sweep of the material model (Eq. 3, Sec. IV's
// comparison over alpha).
//
// k_trace_tris  one ray per (triangle, sample): from the TX to the centroid
//               of one of the k x k sub-triangles of the triangle's regular
//               subdivision (S = k^2 samples, each standing for area / S).
//               The ray traverses the LBVH like a grid ray (traverse.cuh);
//               the sample is visible when its nearest hit is its own
//               triangle (the exact integer test of the Morton position).
//               Visible samples are appended to the scene's hit list as
//               ray = id * S + s.  Rays run in Morton order of their
//               triangles, so a warp's 32 rays aim at neighbouring faces.
// k_echo_tris   one thread per visible sample: the sample point, its
//               distance and direction in FP64 from the triangle's vertices
//               (no traversal rounding enters them), the solid angle
//               Omega = (area / S) |n . u| / t^2 of the patch it stands for,
//               then the echo per receive antenna as for grid rays (Eq. 1-3
//               as expected lobes, path length of Sec. III-B).
// k_alpha_mix   the IF is linear in alpha (a_j = Omega ((1 - alpha) s_j +
//               alpha l_j) / (t r_j), and d, d-dot do not depend on it), so a
//               sweep synthesises alpha = 0 and alpha = 1 once and forms
//               s(alpha) = s(0) + alpha (s(1) - s(0)) for every alpha.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "rr_internal.cuh"

namespace rr {
namespace {

#include "traverse.cuh"

constexpr int kTrisThreads = 128;

// Barycentric coordinates (b1, b2) (point = v0 + b1 e1 + b2 e2) of sample s
// of k x k: the centroids of the subdivision's "up" cells (i, j), i + j <=
// k - 1, at ((i + 1/3) / k, (j + 1/3) / k), row by row, then of its "down"
// cells, i + j <= k - 2, at ((i + 2/3) / k, (j + 2/3) / k).
__host__ __device__ inline void tri_sample_bary(int k, int s, double &b1, double &b2) {
  const int nup = k * (k + 1) / 2;
  const bool up = s < nup;
  int rem = up ? s : s - nup;
  const int rows = up ? k : k - 1;
  int i = 0;
  while (i < rows && rem >= rows - i) {
    rem -= rows - i;
    ++i;
  }
  const double off = up ? 1.0 / 3.0 : 2.0 / 3.0;
  b1 = (i + off) / k;
  b2 = (rem + off) / k;
}

__global__ void __launch_bounds__(kTrisThreads)
k_trace_tris(const FrameJob J, const RadarDev r, int k, uint32_t *__restrict__ err) {
  const int n = J.hdr->n;
  const int root = J.hdr->root;
  if (n <= 0) return;
  const int S = k * k;
  const int64_t total = (int64_t)n * S;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = warp * 32; base < total; base += nwarps * 32) {
    const int64_t q = base + lane;
    const bool valid = q < total;
    const int pos = valid ? (int)(q / S) : 0;
    const int s = valid ? (int)(q - (int64_t)pos * S) : 0;
    float best_t = INFINITY;
    int best_pos = -1, best_id = 0x7fffffff;
    RayPre rp;
    bool active = false;
    if (valid) {
      const float4 a = __ldg(J.tris + 3 * pos), b = __ldg(J.tris + 3 * pos + 1), c = __ldg(J.tris + 3 * pos + 2);
      double b1, b2;
      tri_sample_bary(k, s, b1, b2);
      const float f1 = (float)b1, f2 = (float)b2;
      const float p[3] = {a.x + f1 * (b.x - a.x) + f2 * (c.x - a.x), a.y + f1 * (b.y - a.y) + f2 * (c.y - a.y),
                          a.z + f1 * (b.z - a.z) + f2 * (c.z - a.z)};
      float d[3] = {p[0] - r.txf[0], p[1] - r.txf[1], p[2] - r.txf[2]};
      const float il = rsqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      d[0] *= il; d[1] *= il; d[2] *= il;
      rp.ox = r.txf[0]; rp.oy = r.txf[1]; rp.oz = r.txf[2];
      rp.ix = safe_inv(d[0]); rp.iy = safe_inv(d[1]); rp.iz = safe_inv(d[2]);
      int kz = 0;
      if (fabsf(d[1]) > fabsf(d[kz])) kz = 1;
      if (fabsf(d[2]) > fabsf(d[kz])) kz = 2;
      int kx = kz == 2 ? 0 : kz + 1, ky = kx == 2 ? 0 : kx + 1;
      if (d[kz] < 0.f) { const int tmp = kx; kx = ky; ky = tmp; }
      rp.kx = kx; rp.ky = ky; rp.kz = kz;
      rp.Sx = d[kx] / d[kz];
      rp.Sy = d[ky] / d[kz];
      rp.Sz = 1.0f / d[kz];
      if (root < 0) tri_test(rp, J.tris, ~root, best_t, best_pos, best_id);
      else active = true;
    }
    traverse_warp(rp, J, n, root, active, best_t, best_pos, best_id, err);
    // visible: the nearest hit is the sample's own triangle
    const bool vis = valid && best_pos == pos;
    const uint32_t mask = __ballot_sync(0xffffffffu, vis);
    if (mask != 0u) {
      const int leader = __ffs(mask) - 1;
      uint32_t hb = 0;
      if (lane == leader) hb = atomicAdd(J.count, (uint32_t)__popc(mask));
      hb = __shfl_sync(0xffffffffu, hb, leader);
      if (vis) {
        const int64_t slot = (int64_t)hb + __popc(mask & ((1u << lane) - 1u));
        if (slot < J.cap) {
          J.hit_ray[slot] = best_id * S + s;
          J.hit_tri[slot] = best_id;
          J.hit_pos[slot] = pos;
          J.hit_t[slot] = best_t;
        } else {
          atomicOr(err, ERR_HIT_OVERFLOW);
        }
      }
    }
  }
}

__global__ void __launch_bounds__(128) k_echo_tris(const FrameJob J, const RadarDev r, int k, float alpha) {
  const int S = k * k;
  const int64_t total = min((int64_t)*J.count, J.cap);
  for (int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; h < total; h += (int64_t)gridDim.x * blockDim.x) {
    const int ray = J.hit_ray[h];
    const int pos = J.hit_pos[h];
    const int s = ray % S;
    const float4 fa = __ldg(J.tris + 3 * pos), fb = __ldg(J.tris + 3 * pos + 1), fc = __ldg(J.tris + 3 * pos + 2);
    const double v0[3] = {fa.x, fa.y, fa.z};
    const double e1[3] = {(double)fb.x - v0[0], (double)fb.y - v0[1], (double)fb.z - v0[2]};
    const double e2[3] = {(double)fc.x - v0[0], (double)fc.y - v0[1], (double)fc.z - v0[2]};
    double b1, b2;
    tri_sample_bary(k, s, b1, b2);
    const double p[3] = {v0[0] + b1 * e1[0] + b2 * e2[0], v0[1] + b1 * e1[1] + b2 * e2[1],
                         v0[2] + b1 * e1[2] + b2 * e2[2]};
    const double w0[3] = {p[0] - r.tx[0], p[1] - r.tx[1], p[2] - r.tx[2]};
    const double t = sqrt(w0[0] * w0[0] + w0[1] * w0[1] + w0[2] * w0[2]);
    const double u[3] = {w0[0] / t, w0[1] / t, w0[2] / t};
    const double nn[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    const double nl = sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
    const double un = u[0] * nn[0] + u[1] * nn[1] + u[2] * nn[2];
    J.hit_t[h] = (float)t;
    // unit face normal turned toward the incoming ray (two-sided faces)
    const double sgn = un > 0.0 ? -1.0 / nl : 1.0 / nl;
    const float nf[3] = {(float)(nn[0] * sgn), (float)(nn[1] * sgn), (float)(nn[2] * sgn)};
    const float uf[3] = {(float)u[0], (float)u[1], (float)u[2]};
    const float ci = -(uf[0] * nf[0] + uf[1] * nf[1] + uf[2] * nf[2]);
    const float mr[3] = {uf[0] + 2.f * ci * nf[0], uf[1] + 2.f * ci * nf[1], uf[2] + 2.f * ci * nf[2]};
    // the patch of area / S seen from the TX: its projected area over t^2
    const float omega = (float)(0.5 * fabs(un) / ((double)S * t * t));
    const float tf = (float)t;
    for (int j = 0; j < r.n_rx; ++j) {
      const float wj[3] = {(float)(p[0] - r.rx[j][0]), (float)(p[1] - r.rx[j][1]), (float)(p[2] - r.rx[j][2])};
      const float rj = sqrtf(wj[0] * wj[0] + wj[1] * wj[1] + wj[2] * wj[2]);
      const float irf = 1.f / rj;
      const float uj[3] = {wj[0] * irf, wj[1] * irf, wj[2] * irf};
      const float co = -(uj[0] * nf[0] + uj[1] * nf[1] + uj[2] * nf[2]);
      float gj = 0.f;
      if (co > 0.f) {
        const float sdot = -(mr[0] * uj[0] + mr[1] * uj[1] + mr[2] * uj[2]);
        const float sp = sdot > 0.f ? powf(sdot, r.spec_exp) : 0.f;
        gj = (1.f - alpha) * sp + alpha * (ci * co);
      }
      const int64_t o = (int64_t)j * J.ld + h;
      J.hit_d[o] = (float)(t + (double)rj);
      J.hit_a[o] = r.amp_mode == 1 ? 1.f : omega * gj / (tf * rj);
      J.hit_dd[o] = J.vel[0] * (uf[0] + uj[0]) + J.vel[1] * (uf[1] + uj[1]) + J.vel[2] * (uf[2] + uj[2]);
    }
  }
}

__global__ void k_alpha_mix(const float2 *__restrict__ s0, const float2 *__restrict__ s1, int64_t cube, AlphaList al,
                            float2 *__restrict__ out) {
  const int64_t total = cube * al.n;
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(x / cube);
    const int64_t i = x - (int64_t)a * cube;
    const float2 u = s0[i], v = s1[i];
    const float al_a = al.v[a];
    out[x] = make_float2(fmaf(al_a, v.x - u.x, u.x), fmaf(al_a, v.y - u.y, u.y));
  }
}

int sms() {
  int n = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n;
}

}  // namespace

cudaError_t launch_trace_tris(SceneDev &s, const RadarDev &r, int k, int64_t cap, uint32_t *err, cudaStream_t st) {
  if (k < 1 || k > kMaxTriSide) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(s.hit_count, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  const FrameJob J = frame_job_for(s, GridDev{}, cap);
  const int64_t warps = ((int64_t)s.nt * k * k + 31) / 32;
  const int64_t want = (warps * 32 + kTrisThreads - 1) / kTrisThreads;
  const int blocks = (int)(want < 16 * sms() ? (want < 1 ? 1 : want) : 16 * sms());
  k_trace_tris<<<blocks, kTrisThreads, 0, st>>>(J, r, k, err);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return launch_echo_tris(s, r, k, cap, r.alpha, st);
}

cudaError_t launch_echo_tris(SceneDev &s, const RadarDev &r, int k, int64_t cap, float alpha, cudaStream_t st) {
  const FrameJob J = frame_job_for(s, GridDev{}, cap);
  const int64_t want = (cap + 127) / 128;
  const int blocks = (int)(want < 2 * sms() ? (want < 1 ? 1 : want) : 2 * sms());
  k_echo_tris<<<blocks, 128, 0, st>>>(J, r, k, alpha);
  return cudaGetLastError();
}

cudaError_t launch_alpha_mix(const float *s0, const float *s1, int64_t cube_complex, const AlphaList &al, float *out,
                             cudaStream_t st) {
  const int64_t total = cube_complex * al.n;
  const int64_t want = (total + 255) / 256;
  const int blocks = (int)(want < 8 * sms() ? (want < 1 ? 1 : want) : 8 * sms());
  k_alpha_mix<<<blocks, 256, 0, st>>>(reinterpret_cast<const float2 *>(s0), reinterpret_cast<const float2 *>(s1),
                                      cube_complex, al, reinterpret_cast<float2 *>(out));
  return cudaGetLastError();
}

}  // namespace rr
