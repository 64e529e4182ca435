// imaging.cu -- the imaging workload of Sec. II and IV: the SFCW baseband
// of every TX-RX pair of a MIMO array, its brute-force back-projection into
// a voxel volume and the maximum projection of the volume to a dB image.
//
// k_mimo_geom   one thread per hit of one TX's trace: the FP64 hit point,
//               distance, face normal, mirror direction and solid angle
//               (echo_geometry, the arithmetic of the ray-grid echo).
// k_mimo_sfcw   CTA (RX j, step block, hit split z): each thread computes
//               the echo of one hit at RX j (echo_at_rx: path d = t +
//               |p - rx_j|, amplitude a; the distance then refined to
//               FP64 accuracy) and the hit's phase in cycles,
//               f0 d / c reduced in FP64 plus the per-step term df d / c;
//               then every thread (16 consecutive SFCW steps, one of
//               several hit lanes) adds a exp(-j 2 pi (f0 + n df) d / c)
//               for its share of the block's hits (Eq. 4 with the CW
//               carrier of step n): one sine at the first step, then
//               rotations by the step phasor.  The lanes are summed in a
//               fixed order, hits are split over z for parallelism and
//               k_sfcw_sum adds the splits in a fixed order.
// k_backproject one thread per four voxels: for every TX t and RX j the
//               path R = |v - tx_t| + |v - rx_j| (FP32), the step phasor
//               w = exp(+j 2 pi df R / c), the sum over steps by Horner's
//               rule (sum_n s_n w^n, four FMA per step and voxel), times
//               the carrier exp(+j 2 pi f0 R / c).  The baseband rows are
//               read through L1 by all threads at once (broadcast).  Bound:
//               FP32 FMA issue (ALU).
// k_max_proj / k_db  per (y, x): the largest |I| over z and its index, the
//               volume's maximum by an integer atomic max on the float's
//               bits (non-negative floats order as integers), then dB.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "rr_internal.cuh"

namespace rr {
namespace {

#include "echo_geom.cuh"

struct MimoGeom {
  double p[3];
  double t;
  float nf[3];
  float ci;
  float mr[3];
  float omega;
};
static_assert(sizeof(MimoGeom) == kMimoGeomBytes, "geometry record size");

constexpr int kSfcwThreads = 128;
constexpr int kStepsPerThread = 16;   // SFCW steps per thread: one sine, then phasor rotations
constexpr int kMaxSplits = 64;
constexpr int kBpThreads = 128;
constexpr int kBpVoxels = 4;          // voxels per back-projection thread (independent Horner chains)

__global__ void __launch_bounds__(128) k_mimo_geom(const FrameJob J, const RadarDev r, MimoGeom *__restrict__ geom) {
  const int64_t total = min((int64_t)*J.count, J.cap);
  for (int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; h < total; h += (int64_t)gridDim.x * blockDim.x) {
    const EchoGeom G = echo_geometry(J, r, h);
    MimoGeom m;
    for (int k = 0; k < 3; ++k) {
      m.p[k] = G.p[k];
      m.nf[k] = G.nf[k];
      m.mr[k] = G.mr[k];
    }
    m.t = G.t;
    m.ci = G.ci;
    m.omega = G.omega;
    geom[h] = m;
  }
}

__global__ void __launch_bounds__(kSfcwThreads)
k_mimo_sfcw(const uint32_t *__restrict__ count, int64_t cap, const MimoGeom *__restrict__ geom,
            const double *__restrict__ rx, float alpha, float spec_exp, int amp_mode, double k0, double k1, int n_f,
            int n_rx, int gb, float *__restrict__ part) {
  __shared__ float4 s_h[kSfcwThreads];   // per hit: a, p0, p1 head, p1 tail
  __shared__ float2 s_w[kSfcwThreads];   // per hit: the step phasor (cos, sin)
  __shared__ float2 s_red[kSfcwThreads * kStepsPerThread];
  const int j = blockIdx.x;
  const int lanes = kSfcwThreads / gb;          // hit lanes: threads sharing a step group
  const int gl = threadIdx.x % gb, l = threadIdx.x / gb;
  const int g = blockIdx.y * gb + gl;           // this thread's step group
  const int n_groups = (n_f + kStepsPerThread - 1) / kStepsPerThread;
  const bool active = l < lanes && g < n_groups;
  const float fn0 = (float)(g * kStepsPerThread);
  const int splits = gridDim.z;
  const int64_t total = min((int64_t)*count, cap);
  const double rxj[3] = {rx[3 * j], rx[3 * j + 1], rx[3 * j + 2]};
  float acc_re[kStepsPerThread], acc_im[kStepsPerThread];
#pragma unroll
  for (int i = 0; i < kStepsPerThread; ++i) acc_re[i] = acc_im[i] = 0.f;
  for (int64_t h0 = (int64_t)blockIdx.z * kSfcwThreads; h0 < total; h0 += (int64_t)splits * kSfcwThreads) {
    const int64_t h = h0 + threadIdx.x;
    float a = 0.f, p0 = 0.f, p1h = 0.f, p1l = 0.f, wc = 1.f, ws = 0.f;
    if (h < total) {
      const MimoGeom g = geom[h];
      double d;
      float uj[3];
      echo_at_rx(g.p, g.t, g.nf, g.mr, g.ci, g.omega, rxj, alpha, spec_exp, amp_mode, d, a, uj);
      // the FP32 hit-to-receiver distance refined by one Newton step in
      // FP64 (its rounding alone would be ~1e-5 cycles of phase at 80 GHz)
      {
        const double w0 = g.p[0] - rxj[0], w1 = g.p[1] - rxj[1], w2 = g.p[2] - rxj[2];
        const double r2 = w0 * w0 + w1 * w1 + w2 * w2;
        const double r = d - g.t;
        if (r > 0.0) d = g.t + (r + (r2 - r * r) * (0.5 / r));
      }
      const double c0 = k0 * d;  // cycles of the first carrier, reduced in FP64
      p0 = (float)(c0 - rint(c0));
      // cycles added per step as a 12-bit head, whose product with any
      // step index n < 4096 is exact in FP32 (so its whole cycles drop out
      // exactly), and an FP32 tail; and the step's phasor
      const double c1 = k1 * d;
      p1h = __uint_as_float(__float_as_uint((float)c1) & 0xfffff000u);
      p1l = (float)(c1 - (double)p1h);
      sincospif(2.f * (float)(c1 - rint(c1)), &ws, &wc);
    }
    __syncthreads();
    s_h[threadIdx.x] = make_float4(a, p0, p1h, p1l);
    s_w[threadIdx.x] = make_float2(wc, ws);
    __syncthreads();
    const int m = (int)min((int64_t)kSfcwThreads, total - h0);
    if (active)
      for (int k = l; k < m; k += lanes) {
        // a exp(-j 2 pi phase) at the group's first step, then rotated by
        // the step phasor exp(-j 2 pi df d / c) for the group's other steps
        const float4 hk = s_h[k];
        const float2 wk = s_w[k];
        const float q = fn0 * hk.z;
        float ph = (q - rintf(q)) + fmaf(fn0, hk.w, hk.y);
        ph -= rintf(ph);
        float sn, cs;
        sincospif(2.f * ph, &sn, &cs);
        const float ak = hk.x, c = wk.x, sw = wk.y;
        float zr = ak * cs, zi = -ak * sn;
#pragma unroll
        for (int i = 0; i < kStepsPerThread; ++i) {
          acc_re[i] += zr;
          acc_im[i] += zi;
          const float nr = fmaf(zr, c, zi * sw);
          const float ni = fmaf(zi, c, -zr * sw);
          zr = nr;
          zi = ni;
        }
      }
  }
  // sum over the hit lanes in a fixed order
  __syncthreads();
  if (l < lanes)
#pragma unroll
    for (int i = 0; i < kStepsPerThread; ++i)
      s_red[(l * gb + gl) * kStepsPerThread + i] = make_float2(acc_re[i], acc_im[i]);
  __syncthreads();
  for (int q = threadIdx.x; q < gb * kStepsPerThread; q += blockDim.x) {
    const int qg = q / kStepsPerThread, i = q % kStepsPerThread;
    const int n = (blockIdx.y * gb + qg) * kStepsPerThread + i;
    float re = 0.f, im = 0.f;
    for (int ll = 0; ll < lanes; ++ll) {
      const float2 v = s_red[(ll * gb + qg) * kStepsPerThread + i];
      re += v.x;
      im += v.y;
    }
    if (n < n_f) {
      float *o = part + (((int64_t)blockIdx.z * n_rx + j) * n_f + n) * 2;
      o[0] = re;
      o[1] = im;
    }
  }
}

__global__ void k_sfcw_sum(const float2 *__restrict__ part, int splits, int64_t n, float2 *__restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float re = 0.f, im = 0.f;
    for (int z = 0; z < splits; ++z) {
      const float2 v = part[z * n + i];
      re += v.x;
      im += v.y;
    }
    out[i] = make_float2(re, im);
  }
}

// Cycles of k R for k = kh + kl (kh the float nearest k): the product's
// rounding error is recovered with an FMA, so the phase keeps the accuracy
// of R itself.
__device__ __forceinline__ float cycles_of(float kh, float kl, float R) {
  const float p = kh * R;
  const float e = fmaf(kh, R, -p);
  return (p - rintf(p)) + fmaf(kl, R, e);
}

// One Horner step acc = acc w + s for each of the thread's voxels.
template <int V>
__device__ __forceinline__ void horner_step(float (&ar)[V], float (&ai)[V], const float (&wr)[V], const float (&wi)[V],
                                            float sr, float si) {
#pragma unroll
  for (int k = 0; k < V; ++k) {
    const float tr = fmaf(ar[k], wr[k], fmaf(-ai[k], wi[k], sr));
    const float ti = fmaf(ar[k], wi[k], fmaf(ai[k], wr[k], si));
    ar[k] = tr;
    ai[k] = ti;
  }
}

// PAIRS: the rows are read two steps at a time (16-byte loads; n_f even
// and s 16-byte aligned).
template <bool PAIRS>
__global__ void __launch_bounds__(kBpThreads)
k_backproject(const float2 *__restrict__ s, const float4 *__restrict__ pos, int n_tx, int n_rx, float k0h, float k0l,
              float k1h, float k1l, int n_f, const VolumeDev v, float2 *__restrict__ img) {
  constexpr int V = kBpVoxels;
  extern __shared__ float4 s_pos[];
  for (int i = threadIdx.x; i < n_tx + n_rx; i += blockDim.x) s_pos[i] = pos[i];
  __syncthreads();
  const int64_t nvox = (int64_t)v.nx * v.ny * v.nz;
  const int64_t i0 = ((int64_t)blockIdx.x * kBpThreads + threadIdx.x) * V;
  float vx[V], vy[V], vz[V];
#pragma unroll
  for (int k = 0; k < V; ++k) {
    const int64_t i = min(i0 + k, nvox - 1);
    const int ix = (int)(i % v.nx);
    const int iy = (int)((i / v.nx) % v.ny);
    const int iz = (int)(i / ((int64_t)v.nx * v.ny));
    vx[k] = fmaf((float)ix, v.dx, v.x0);
    vy[k] = fmaf((float)iy, v.dy, v.y0);
    vz[k] = fmaf((float)iz, v.dz, v.z0);
  }
  float ir[V], ii[V];
#pragma unroll
  for (int k = 0; k < V; ++k) ir[k] = ii[k] = 0.f;
  for (int t = 0; t < n_tx; ++t) {
    const float4 T = s_pos[t];
    float dt[V];
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const float a = vx[k] - T.x, b = vy[k] - T.y, c = vz[k] - T.z;
      dt[k] = sqrtf(fmaf(a, a, fmaf(b, b, c * c)));
    }
    const float2 *srow = s + (int64_t)t * n_rx * n_f;
    for (int j = 0; j < n_rx; ++j, srow += n_f) {
      const float4 Q = s_pos[n_tx + j];
      float R[V], wr[V], wi[V], ar[V], ai[V];
#pragma unroll
      for (int k = 0; k < V; ++k) {
        const float a = vx[k] - Q.x, b = vy[k] - Q.y, c = vz[k] - Q.z;
        R[k] = dt[k] + sqrtf(fmaf(a, a, fmaf(b, b, c * c)));
        sincospif(2.f * cycles_of(k1h, k1l, R[k]), &wi[k], &wr[k]);
        ar[k] = 0.f;
        ai[k] = 0.f;
      }
      // sum_n s_n w^n by Horner's rule, highest step first
      if (PAIRS) {
        const float4 *s4 = reinterpret_cast<const float4 *>(srow);
#pragma unroll 4
        for (int q = n_f / 2 - 1; q >= 0; --q) {
          const float4 sv = __ldg(s4 + q);  // steps 2q, 2q + 1
          horner_step<V>(ar, ai, wr, wi, sv.z, sv.w);
          horner_step<V>(ar, ai, wr, wi, sv.x, sv.y);
        }
      } else {
#pragma unroll 8
        for (int n = n_f - 1; n >= 0; --n) {
          const float2 sv = __ldg(srow + n);
          horner_step<V>(ar, ai, wr, wi, sv.x, sv.y);
        }
      }
#pragma unroll
      for (int k = 0; k < V; ++k) {
        float sn, cs;
        sincospif(2.f * cycles_of(k0h, k0l, R[k]), &sn, &cs);
        ir[k] = fmaf(ar[k], cs, fmaf(-ai[k], sn, ir[k]));
        ii[k] = fmaf(ar[k], sn, fmaf(ai[k], cs, ii[k]));
      }
    }
  }
#pragma unroll
  for (int k = 0; k < V; ++k)
    if (i0 + k < nvox) img[i0 + k] = make_float2(ir[k], ii[k]);
}

__global__ void k_max_proj(const float2 *__restrict__ img, const VolumeDev v, float *__restrict__ amp,
                           int32_t *__restrict__ zi, uint32_t *__restrict__ gmax) {
  const int64_t plane = (int64_t)v.nx * v.ny;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < plane; i += (int64_t)gridDim.x * blockDim.x) {
    float best = -1.f;
    int bz = 0;
    for (int z = 0; z < v.nz; ++z) {
      const float2 x = img[z * plane + i];
      const float a = sqrtf(x.x * x.x + x.y * x.y);
      if (a > best) {
        best = a;
        bz = z;
      }
    }
    amp[i] = best;
    if (zi) zi[i] = bz;
    atomicMax(gmax, __float_as_uint(best));
  }
}

__global__ void k_db(const float *__restrict__ amp, int64_t n, const uint32_t *__restrict__ gmax, float dyn_db,
                     float *__restrict__ db) {
  const float top = __uint_as_float(*gmax);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float x = top > 0.f ? 20.f * log10f(amp[i] / top) : -INFINITY;
    db[i] = fmaxf(x, -dyn_db);
  }
}

int sms() {
  int n = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n;
}

void split_double(double x, float &hi, float &lo) {
  hi = (float)x;
  lo = (float)(x - (double)hi);
}

}  // namespace

// Step groups per CTA (the rest of its threads take other hits).
int mimo_sfcw_groups(int n_f) {
  const int n_groups = (n_f + kStepsPerThread - 1) / kStepsPerThread;
  return n_groups < kSfcwThreads ? n_groups : kSfcwThreads;
}

int mimo_sfcw_splits(int n_rx, int n_f) {
  const int gb = mimo_sfcw_groups(n_f);
  const int ctas = n_rx * (((n_f + kStepsPerThread - 1) / kStepsPerThread + gb - 1) / gb);
  int z = (4 * sms() + ctas - 1) / ctas;
  return z < 1 ? 1 : (z > kMaxSplits ? kMaxSplits : z);
}

cudaError_t launch_mimo_sfcw(SceneDev &s, const RadarDev &r, const GridDev &g, int64_t cap, double2 *dir,
                             const double *rx, int n_rx, double f0, double df, int n_f, void *geom, float *part,
                             float *out, cudaStream_t st) {
  FrameJob J = frame_job_for(s, g, cap);
  J.dir = dir;
  const int n_sm = sms();
  k_mimo_geom<<<4 * n_sm, 128, 0, st>>>(J, r, static_cast<MimoGeom *>(geom));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const double c = 299792458.0;
  const int zs = mimo_sfcw_splits(n_rx, n_f);
  const int gb = mimo_sfcw_groups(n_f);
  const int n_groups = (n_f + kStepsPerThread - 1) / kStepsPerThread;
  const dim3 grid(n_rx, (n_groups + gb - 1) / gb, zs);
  k_mimo_sfcw<<<grid, kSfcwThreads, 0, st>>>(s.hit_count, cap, static_cast<const MimoGeom *>(geom), rx, r.alpha,
                                             r.spec_exp, r.amp_mode, f0 / c, df / c, n_f, n_rx, gb, part);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int64_t n = (int64_t)n_rx * n_f;
  k_sfcw_sum<<<(int)((n + 255) / 256 < 4 * n_sm ? (n + 255) / 256 : 4 * n_sm), 256, 0, st>>>(
      reinterpret_cast<const float2 *>(part), zs, n, reinterpret_cast<float2 *>(out));
  return cudaGetLastError();
}

cudaError_t launch_backproject(const float *s, const float4 *pos, int n_tx, int n_rx, double f0, double df, int n_f,
                               const VolumeDev &v, float *img, cudaStream_t st) {
  const int64_t nvox = (int64_t)v.nx * v.ny * v.nz;
  if (nvox <= 0) return cudaSuccess;
  const double c = 299792458.0;
  float k0h, k0l, k1h, k1l;
  split_double(f0 / c, k0h, k0l);
  split_double(df / c, k1h, k1l);
  const size_t smem = sizeof(float4) * (size_t)(n_tx + n_rx);
  const bool pairs = n_f % 2 == 0 && reinterpret_cast<uintptr_t>(s) % 16 == 0;
  if (smem > 48 * 1024) {
    cudaError_t e = pairs ? cudaFuncSetAttribute(k_backproject<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                          : cudaFuncSetAttribute(k_backproject<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int64_t per = (int64_t)kBpVoxels * kBpThreads;
  const unsigned blocks = (unsigned)((nvox + per - 1) / per);
  const float2 *s2 = reinterpret_cast<const float2 *>(s);
  float2 *o = reinterpret_cast<float2 *>(img);
  if (pairs)
    k_backproject<true><<<blocks, kBpThreads, smem, st>>>(s2, pos, n_tx, n_rx, k0h, k0l, k1h, k1l, n_f, v, o);
  else
    k_backproject<false><<<blocks, kBpThreads, smem, st>>>(s2, pos, n_tx, n_rx, k0h, k0l, k1h, k1l, n_f, v, o);
  return cudaGetLastError();
}

cudaError_t launch_max_projection(const float *img, const VolumeDev &v, float dyn_db, float *db, int32_t *z,
                                  float *amp_tmp, uint32_t *gmax, cudaStream_t st) {
  const int64_t plane = (int64_t)v.nx * v.ny;
  if (plane <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(gmax, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  const int n_sm = sms();
  const int blocks = (int)((plane + 255) / 256 < 4 * n_sm ? (plane + 255) / 256 : 4 * n_sm);
  k_max_proj<<<blocks, 256, 0, st>>>(reinterpret_cast<const float2 *>(img), v, amp_tmp, z, gmax);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_db<<<blocks, 256, 0, st>>>(amp_tmp, plane, gmax, dyn_db, db);
  return cudaGetLastError();
}

}  // namespace rr
