// stochastic.cu -- the material model of Eq. 1-3 as the paper states it
// (Sec. III-A: a random diffuse direction n + r, r a random point on the
// unit sphere, mixed with the mirror direction by alpha), with reception
// cones at the antennas, return-leg occlusion and multiple bounces.
//
// k_trace_stochastic  a warp takes 32 consecutive rays of the grid; every
//                     lane walks its ray through up to B bounces, all lanes
//                     in step so that each traversal (closest hit, then one
//                     return leg per antenna) is one warp-uniform walk
//                     (traverse.cuh).  At a hit the random unit vector comes
//                     from Philox4x32-10 (counter (ray, bounce, 0, 0), key
//                     (seed, frame): the same stream whatever the launch
//                     shape), the outgoing direction is the normalised mix
//                     of Eq. 3, and antenna j receives when that direction
//                     lies within theta_r of the direction to it, the
//                     antenna is in front of the face and the return leg
//                     is free.  A bounce with a receiving antenna is one
//                     hit-list entry: path length d_j = legs + |rx_j - p|,
//                     amplitude Omega / (2 pi (1 - cos theta_r)) per
//                     receiving antenna (0 for the others), path rate
//                     v . (u_0 - w_j).  Bounce and return-leg rays start
//                     kStochEps along the facing normal.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "rr_internal.cuh"

namespace rr {
namespace {

#include "traverse.cuh"

constexpr int kStochThreads = 128;

// Philox4x32-10 (Salmon et al., SC 2011) from its published definition.
__device__ __forceinline__ uint4 philox4x32(uint4 c, uint2 k) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ void make_ray(RayPre &rp, const float o[3], const float d[3]) {
  rp.ox = o[0]; rp.oy = o[1]; rp.oz = o[2];
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
}

__global__ void __launch_bounds__(kStochThreads)
k_trace_stochastic(const FrameJob J, const RadarDev r, const StochParams sp, uint32_t *__restrict__ err) {
  const int n = J.hdr->n;
  const int root = J.hdr->root;
  if (n <= 0) return;
  const int64_t total = (int64_t)J.g.n_az * J.g.n_el;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const float cos_r = cosf(sp.theta_r);
  const float amp = r.amp_mode == 1 ? 1.f : 0.f;  // set per ray below otherwise
  for (int64_t base = warp * 32; base < total; base += nwarps * 32) {
    const int64_t q = base + lane;
    bool alive = q < total;
    const int ray = alive ? (int)q : 0;
    const int i_el = ray / J.g.n_az, i_az = ray - i_el * J.g.n_az;
    float u[3] = {0.f, 0.f, 1.f}, o[3] = {r.txf[0], r.txf[1], r.txf[2]};
    float a_recv = amp;
    if (alive) {
      float sa, ca, se, ce;
      sincospif(fmaf((float)i_az, J.g.daz_pi, J.g.az0_pi), &sa, &ca);
      sincospif(fmaf((float)i_el, J.g.del_pi, J.g.el0_pi), &se, &ce);
      const float ur[3] = {ce * sa, se, ce * ca};
#pragma unroll
      for (int k = 0; k < 3; ++k) u[k] = r.Rf[3 * k] * ur[0] + r.Rf[3 * k + 1] * ur[1] + r.Rf[3 * k + 2] * ur[2];
      if (r.amp_mode != 1) a_recv = ce * J.g.daz_f * J.g.del_f / (6.2831853f * (1.f - cos_r));
    }
    const float u0[3] = {u[0], u[1], u[2]};
    double legs = 0.0;
    for (int b = 0; b < sp.bounces; ++b) {
      if (!__any_sync(0xffffffffu, alive)) break;
      RayPre rp;
      make_ray(rp, o, u);
      float best_t = INFINITY;
      int best_pos = -1, best_id = 0x7fffffff;
      if (alive && root < 0) tri_test(rp, J.tris, ~root, best_t, best_pos, best_id);
      traverse_warp(rp, J, n, root, alive && root >= 0, best_t, best_pos, best_id, err);
      const bool hit = alive && best_pos >= 0;
      float p[3] = {0.f, 0.f, 0.f}, nf[3] = {0.f, 0.f, 1.f}, tc[3] = {0.f, 0.f, 1.f}, qo[3] = {0.f, 0.f, 0.f};
      if (hit) {
        legs += (double)best_t;
        for (int k = 0; k < 3; ++k) p[k] = o[k] + best_t * u[k];
        const float4 fa = __ldg(J.tris + 3 * best_pos), fb = __ldg(J.tris + 3 * best_pos + 1),
                     fc = __ldg(J.tris + 3 * best_pos + 2);
        const float e1[3] = {fb.x - fa.x, fb.y - fa.y, fb.z - fa.z}, e2[3] = {fc.x - fa.x, fc.y - fa.y, fc.z - fa.z};
        const float nn[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        const float nl = sqrtf(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
        const float un = u[0] * nn[0] + u[1] * nn[1] + u[2] * nn[2];
        const float sg = un > 0.f ? -1.f / nl : 1.f / nl;
        for (int k = 0; k < 3; ++k) nf[k] = nn[k] * sg;
        // Eq. 1: a random point on the unit sphere (FP64 from the 32-bit words)
        const uint4 x = philox4x32(make_uint4((uint32_t)ray, (uint32_t)b, 0u, 0u), make_uint2(sp.seed, sp.frame));
        const double u1 = ((double)x.x + 0.5) * 2.3283064365386963e-10, u2 = ((double)x.y + 0.5) * 2.3283064365386963e-10;
        const double z = 1.0 - 2.0 * u1, s = sqrt(fmax(0.0, 1.0 - z * z));
        double sp_, cp_;
        sincospi(2.0 * u2, &sp_, &cp_);
        float td[3] = {nf[0] + (float)(s * cp_), nf[1] + (float)(s * sp_), nf[2] + (float)z};
        float l = sqrtf(td[0] * td[0] + td[1] * td[1] + td[2] * td[2]);
        for (int k = 0; k < 3; ++k) td[k] = l > 0.f ? td[k] / l : nf[k];
        // Eq. 2: mirror direction; Eq. 3: the normalised mix
        const float c2 = 2.f * (u[0] * nf[0] + u[1] * nf[1] + u[2] * nf[2]);
        for (int k = 0; k < 3; ++k) tc[k] = sp.alpha * td[k] + (1.f - sp.alpha) * (u[k] - c2 * nf[k]);
        l = sqrtf(tc[0] * tc[0] + tc[1] * tc[1] + tc[2] * tc[2]);
        for (int k = 0; k < 3; ++k) tc[k] = l > 0.f ? tc[k] / l : nf[k];
        for (int k = 0; k < 3; ++k) qo[k] = p[k] + kStochEps * nf[k];
      }
      // reception: one return-leg walk per antenna
      float dj[RR_MAX_RX], aj[RR_MAX_RX], ddj[RR_MAX_RX];
      bool any = false;
      for (int j = 0; j < r.n_rx; ++j) {
        const float rxj[3] = {(float)r.rx[j][0], (float)r.rx[j][1], (float)r.rx[j][2]};
        const float w[3] = {rxj[0] - p[0], rxj[1] - p[1], rxj[2] - p[2]};
        const float L = sqrtf(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
        const float wu[3] = {w[0] / L, w[1] / L, w[2] / L};
        dj[j] = (float)(legs + (double)L);
        ddj[j] = J.vel[0] * (u0[0] - wu[0]) + J.vel[1] * (u0[1] - wu[1]) + J.vel[2] * (u0[2] - wu[2]);
        aj[j] = 0.f;
        const bool cand = hit && (tc[0] * wu[0] + tc[1] * wu[1] + tc[2] * wu[2]) >= cos_r &&
                          (wu[0] * nf[0] + wu[1] * nf[1] + wu[2] * nf[2]) > 0.f;
        float ws[3] = {rxj[0] - qo[0], rxj[1] - qo[1], rxj[2] - qo[2]};
        const float Ls = sqrtf(ws[0] * ws[0] + ws[1] * ws[1] + ws[2] * ws[2]);
        for (int k = 0; k < 3; ++k) ws[k] = cand ? ws[k] / Ls : (k == 2 ? 1.f : 0.f);
        RayPre rs;
        make_ray(rs, cand ? qo : o, ws);
        float st = cand ? Ls : 0.f;
        int sp_pos = -1, sp_id = 0x7fffffff;
        if (__any_sync(0xffffffffu, cand)) {
          if (cand && root < 0) tri_test(rs, J.tris, ~root, st, sp_pos, sp_id);
          traverse_warp(rs, J, n, root, cand && root >= 0, st, sp_pos, sp_id, err);
        }
        if (cand && sp_pos < 0) {
          aj[j] = a_recv;
          any = true;
        }
      }
      const uint32_t mask = __ballot_sync(0xffffffffu, any);
      if (mask != 0u) {
        const int leader = __ffs(mask) - 1;
        uint32_t hb = 0;
        if (lane == leader) hb = atomicAdd(J.count, (uint32_t)__popc(mask));
        hb = __shfl_sync(0xffffffffu, hb, leader);
        if (any) {
          const int64_t slot = (int64_t)hb + __popc(mask & ((1u << lane) - 1u));
          if (slot < J.cap) {
            J.hit_ray[slot] = ray * sp.bounces + b;  // unique per entry
            J.hit_tri[slot] = best_id;
            J.hit_pos[slot] = b;
            J.hit_t[slot] = (float)legs;
            for (int j = 0; j < r.n_rx; ++j) {
              const int64_t oo = (int64_t)j * J.ld + slot;
              J.hit_d[oo] = dj[j];
              J.hit_a[oo] = aj[j];
              J.hit_dd[oo] = ddj[j];
            }
          } else {
            atomicOr(err, ERR_HIT_OVERFLOW);
          }
        }
      }
      alive = hit;
      for (int k = 0; k < 3; ++k) {
        o[k] = hit ? qo[k] : o[k];
        u[k] = hit ? tc[k] : u[k];
      }
    }
  }
}

// Philox words for the device check: out[4 i + w] = word w of counter (i, c1, 0, 0), key (k0, k1).
__global__ void k_philox_words(uint32_t k0, uint32_t k1, uint32_t c1, int64_t n, uint32_t *out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint4 x = philox4x32(make_uint4((uint32_t)i, c1, 0u, 0u), make_uint2(k0, k1));
    out[4 * i] = x.x;
    out[4 * i + 1] = x.y;
    out[4 * i + 2] = x.z;
    out[4 * i + 3] = x.w;
  }
}

}  // namespace

cudaError_t launch_trace_stochastic(SceneDev &s, const RadarDev &r, const GridDev &g, const StochParams &sp,
                                    int64_t cap, uint32_t *err, cudaStream_t st) {
  if (sp.bounces < 1 || sp.bounces > kMaxBounces) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(s.hit_count, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  const FrameJob J = frame_job_for(s, g, cap);
  int sms = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = ((int64_t)g.n_az * g.n_el + kStochThreads - 1) / kStochThreads;
  const int blocks = (int)(want < 16 * sms ? (want < 1 ? 1 : want) : 16 * sms);
  k_trace_stochastic<<<blocks, kStochThreads, 0, st>>>(J, r, sp, err);
  return cudaGetLastError();
}

cudaError_t launch_philox_words(uint32_t k0, uint32_t k1, uint32_t c1, int64_t n, uint32_t *out, cudaStream_t st) {
  const int64_t want = (n + 255) / 256;
  k_philox_words<<<(int)(want < 1024 ? (want < 1 ? 1 : want) : 1024), 256, 0, st>>>(k0, k1, c1, n, out);
  return cudaGetLastError();
}

}  // namespace rr
