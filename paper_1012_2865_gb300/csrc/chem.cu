// chem.cu -- per-cell kernels around the trace: the hydrogen-only ionisation
// update (Eq. "dndt", Step 6 of Sec. 3.1), the absorber-density refresh
// n_HI = n_H x_HI, and conversion of the rates for the caller.
#include <cuda_runtime.h>
#include <stdint.h>

#include "f2.cuh"
#include "rt_internal.cuh"

namespace rtg {

// One cell, FP64 path: the backward-Euler substeps below, explicitly rounded.
__device__ __forceinline__ void chem_cell_fp64(double& x, double& z, double n, double kc, double h, int nsub,
                                               double alpha) {
  const double a = __dmul_rn(__dmul_rn(h, alpha), n);
  const double hk = __dmul_rn(h, kc);
  const double b = __dadd_rn(1.0, hk);
  for (int i = 0; i < nsub; ++i) {
    const double D = __dadd_rn(__dmul_rn(b, b), __dmul_rn(__dmul_rn(4.0, a), __dadd_rn(z, hk)));
    const double sq = __dsqrt_rn(D);
    const double xn = __ddiv_rn(__dmul_rn(2.0, __dadd_rn(a, x)), __dadd_rn(__dadd_rn(__dmul_rn(2.0, a), b), sq));
    const double zn = __ddiv_rn(__dmul_rn(2.0, __dadd_rn(z, hk)), __dadd_rn(b, sq));
    if (xn <= zn) { x = xn; z = __dsub_rn(1.0, xn); }
    else { z = zn; x = __dsub_rn(1.0, zn); }
  }
}

// x == 1 and z == 0 (either sign), compared as bit patterns
__device__ __forceinline__ bool is_neutral(double x, double z) {
  return __double_as_longlong(x) == 0x3FF0000000000000LL && (__double_as_longlong(z) << 1) == 0;
}

// One cell, FP32-mixed path: FP32 solution + one double-float Newton
// correction per substep (see chem_mixed_kernel).  x, z and n arrive and
// leave in FP64 (converted through their bit fields, off the FP64 pipe); in
// between, the smaller of the two fractions is carried as a double-float
// pair s and the larger only as its FP32 complement until a substep needs it
// as a pair.  ha and h2 are h alpha_B and h as pairs.  Returns
// n_HI = n_H x_HI as a pair.
__device__ __forceinline__ F2 chem_cell_mixed(double& x, double& z, double n, float kc, F2 ha, F2 h2, int nsub) {
  const F2 n2 = f2_from_double_bits(n);
  const F2 a = f2_mul(ha, n2);
  const F2 hk = f2_mul_f(h2, kc);
  const F2 one = {1.0f, 0.0f};
  const F2 b = f2_add(one, hk);
  const F2 two_a_b = f2_add(F2{2.0f * a.hi, 2.0f * a.lo}, b);
  const float af = a.hi, bf = b.hi, hkf = hk.hi;
  const F2 x0 = f2_from_double_bits(x), z0 = f2_from_double_bits(z);
  float xf = x0.hi, zf = z0.hi;
  bool sx = xf < 0.5f;  // s holds x_HI (else x_HII)
  F2 s = sx ? x0 : z0;
  for (int i = 0; i < nsub; ++i) {
    const float wf = zf + hkf;
    // the FP32 guess needs only ~1e-7: approximate square root and quotient
    // (D >= 1 and both denominators >= 2); the correction's quotient is exact
    const float D = fmaf(4.0f * af, wf, bf * bf);
    const float sq = D * rsqrtf(D);
    if (xf < 0.5f) {
      if (!sx) {
        s = f2_sub(one, s);
        sx = true;
      }
      const float xg = __fdividef(2.0f * (af + xf), 2.0f * af + bf + sq);
      const F2 t = f2_mul_f(f2_sub(f2_mul_f(a, xg), two_a_b), xg);
      const float g = f2_sum_float(t, f2_add(a, s));
      const float gp = fmaf(2.0f * af, xg, -(2.0f * af + bf));
      s = two_sum(xg, -__fdiv_rn(g, gp));
      xf = s.hi;
      zf = 1.0f - xf;
    } else {
      if (sx) {
        s = f2_sub(one, s);
        sx = false;
      }
      const float zg = __fdividef(2.0f * wf, bf + sq);
      const F2 t = f2_mul_f(f2_add(f2_mul_f(a, zg), b), zg);
      const F2 c = f2_add(s, hk);
      const float f = f2_sum_float(t, F2{-c.hi, -c.lo});
      const float fp = fmaf(2.0f * af, zg, bf);
      s = two_sum(zg, -__fdiv_rn(f, fp));
      zf = s.hi;
      xf = 1.0f - zf;
    }
  }
  const F2 xp = sx ? s : f2_sub(one, s);
  const F2 zp = sx ? f2_sub(one, s) : s;
  x = f2_to_double_bits(xp);
  z = f2_to_double_bits(zp);
  return f2_mul(n2, xp);
}

// Backward Euler on dx/dt = alpha_B n_H (1 - x)^2 - k x, x = x_HI,
// z = x_HII, over nsub substeps h with k frozen.  With a = h alpha_B n_H and
// b = 1 + h k the implicit step solves a x'^2 - (2a + b) x' + (a + x) = 0;
// its physical root, written without cancellation, is
//   x' = 2(a + x) / (2a + b + sqrt(D)),  z' = 2(z + hk) / (b + sqrt(D)),
//   D = b^2 + 4a(z + hk),
// and the smaller of x', z' is kept with the other as its complement, so both
// fractions keep their relative accuracy as either tends to 0.  All FP64,
// explicitly rounded (no FMA contraction).
template <typename KT, typename NT>
__global__ void chem_kernel(long long ncell, const double* __restrict__ nH, double* __restrict__ xHI,
                            double* __restrict__ xHII, const KT* __restrict__ K, NT* __restrict__ nhi,
                            double h, int nsub, double alpha) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    double x = xHI[c], z = xHII[c];
    const KT kc = K[c];
    // no radiation and fully neutral: every substep returns (1, 0) exactly
    if (kc == (KT)0 && z == 0.0 && x == 1.0) continue;
    const double n = nH[c];
    chem_cell_fp64(x, z, n, (double)kc, h, nsub, alpha);
    xHI[c] = x;
    xHII[c] = z;
    nhi[c] = (NT)__dmul_rn(n, x);
  }
}

// Same backward-Euler step for the FP32-mixed path, solved by FP32 + one
// Newton correction: the smaller fraction is first obtained in FP32 from its
// cancellation-free formula, then corrected once with the residual of the
// implicit equation evaluated in double-float arithmetic,
//   x-form: g(x') = a x'^2 - (2a + b) x' + (a + x),  g' = 2a x' - (2a + b),
//   z-form: f(z') = a z'^2 + b z' - (z + hk),         f' = 2a z' + b.
// From a ~1e-7 relative guess one Newton step leaves ~1e-14 (the residual's
// double-float rounding, ~2^-48 of its largest term), so the carried state
// stays within ~1e-13 of the FP64 recursion while the substeps run on the
// FP32 pipe.  FP64 arithmetic is left only in one addition per stored
// fraction: the state's conversions to and from pairs move bit fields
// (f2.cuh), since the FP64 pipe, a small fraction of the FP32 one, otherwise
// bounds the kernel.
__global__ void chem_mixed_kernel(long long ncell, const double* __restrict__ nH, double* __restrict__ xHI,
                                  double* __restrict__ xHII, const float* __restrict__ K,
                                  float2* __restrict__ nhi, float4 hh, int nsub) {
  const F2 ha = {hh.x, hh.y}, h2 = {hh.z, hh.w};
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    double x = xHI[c], z = xHII[c];
    const float kc = K[c];
    if (kc == 0.0f && is_neutral(x, z)) continue;
    const F2 nx = chem_cell_mixed(x, z, nH[c], kc, ha, h2, nsub);
    xHI[c] = x;
    xHII[c] = z;
    nhi[c] = make_float2(nx.hi, nx.lo);
  }
}

template <typename NT>
__global__ void refresh_nhi_kernel(long long ncell, const double* __restrict__ nH,
                                   const double* __restrict__ xHI, NT* __restrict__ nhi) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x)
    nhi[c] = (NT)__dmul_rn(nH[c], xHI[c]);
}

// FP32-mixed grids keep n_HI as a pair: FP32 rounding and remainder of the
// FP64 product.
__global__ void refresh_nhi_pair_kernel(long long ncell, const double* __restrict__ nH,
                                        const double* __restrict__ xHI, float2* __restrict__ nhi) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    const F2 v = f2_from_double(__dmul_rn(nH[c], xHI[c]));
    nhi[c] = make_float2(v.hi, v.lo);
  }
}

// FP32 pairs (rounded value, remainder) of an FP64 absorber density.
__global__ void pair_kernel(long long ncell, const double* __restrict__ src, float2* __restrict__ dst) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    const F2 v = f2_from_double(src[c]);
    dst[c] = make_float2(v.hi, v.lo);
  }
}

// First cell whose density is negative, NaN or infinite (atomicMin into bad).
__global__ void check_density_kernel(long long n, const double* __restrict__ a, unsigned long long* __restrict__ bad) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const double v = a[c];
    if (!(v >= 0.0) || isinf(v)) atomicMin(bad, (unsigned long long)c);
  }
}

template <typename ST, typename DT>
__global__ void convert_kernel(long long n, const ST* __restrict__ src, DT* __restrict__ dst, double scale) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x)
    dst[c] = scale == 1.0 ? (DT)src[c] : (DT)((double)src[c] * scale);
}

__global__ void complement_kernel(long long n, const double* __restrict__ x, double* __restrict__ out) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x)
    out[c] = __dsub_rn(1.0, x[c]);
}

// Range check of a gas state: bad[0] = first cell whose n_H is negative, NaN
// or infinite (nH may be NULL), bad[1] = first cell whose x_HI lies outside
// [0, 1] or is NaN; entries stay at ~0 when every cell passes.
__global__ void check_state_kernel(long long n, const double* __restrict__ nH, const double* __restrict__ x,
                                   unsigned long long* __restrict__ bad) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    if (nH) {
      const double v = nH[c];
      if (!(v >= 0.0) || isinf(v)) atomicMin(&bad[0], (unsigned long long)c);
    }
    const double xv = x[c];
    if (!(xv >= 0.0 && xv <= 1.0)) atomicMin(&bad[1], (unsigned long long)c);
  }
}

// The same check two cells at a time (16-byte loads, twice the bytes in
// flight per thread), for 16-byte aligned arrays of an even length.
__global__ void check_state2_kernel(long long n2, const double2* __restrict__ nH, const double2* __restrict__ x,
                                    unsigned long long* __restrict__ bad) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
    if (nH) {
      const double2 v = nH[i];
      if (!(v.x >= 0.0) || isinf(v.x)) atomicMin(&bad[0], (unsigned long long)(2 * i));
      if (!(v.y >= 0.0) || isinf(v.y)) atomicMin(&bad[0], (unsigned long long)(2 * i + 1));
    }
    const double2 xv = x[i];
    if (!(xv.x >= 0.0 && xv.x <= 1.0)) atomicMin(&bad[1], (unsigned long long)(2 * i));
    if (!(xv.y >= 0.0 && xv.y <= 1.0)) atomicMin(&bad[1], (unsigned long long)(2 * i + 1));
  }
}

// Commit of a gas state uploaded without waiting (rt_set_state_async), run
// after check_state_kernel has left the first failing cells in
// ctl[CTL_CHECK_N] and ctl[CTL_CHECK_X] (~0 = none).  When every cell passed,
// the staged arrays replace the grid's -- n_H only when sn is given, x_HII
// from sz or as 1 - x_HI -- and the absorber density n_HI = n_H x_HI is
// refreshed (FP64, or the FP32 pair on the mixed path).  Otherwise nothing
// changes and the rejection is latched in ctl[CTL_SET_ERR] (the first one
// keeps its failing cells), where the next trace and rt_synchronize find it.
// The block that finishes last (CTL_COMMIT_DONE) sets the check words back
// to ~0 for the next upload, after every block has read them.
__device__ __forceinline__ bool commit_verdict(unsigned long long* ctl) {
  const unsigned long long bn = ctl[CTL_CHECK_N], bx = ctl[CTL_CHECK_X];
  if (bn == ~0ULL && bx == ~0ULL) return true;
  if (blockIdx.x == 0 && threadIdx.x == 0 &&
      atomicCAS(&ctl[CTL_SET_ERR], 0ULL, (unsigned long long)RT_ERR_INVALID_ARG) == 0ULL) {
    ctl[CTL_SET_BADN] = bn;
    ctl[CTL_SET_BADX] = bx;
  }
  return false;
}
__device__ __forceinline__ void commit_finish(unsigned long long* ctl) {
  __shared__ int last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&ctl[CTL_COMMIT_DONE], 1ULL) == (unsigned long long)gridDim.x - 1ULL;
    if (last) {
      __threadfence();
      ctl[CTL_CHECK_N] = ~0ULL;
      ctl[CTL_CHECK_X] = ~0ULL;
      ctl[CTL_COMMIT_DONE] = 0ULL;
    }
  }
}
template <bool PAIR>
__global__ void commit_state_kernel(long long n, unsigned long long* __restrict__ ctl, const double* __restrict__ sn,
                                    const double* __restrict__ sx, const double* __restrict__ sz,
                                    double* __restrict__ nH, double* __restrict__ xHI, double* __restrict__ xHII,
                                    void* __restrict__ nhi) {
  const bool ok = commit_verdict(ctl);
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; ok && c < n;
       c += (long long)gridDim.x * blockDim.x) {
    const double h = sn ? sn[c] : nH[c];
    if (sn) nH[c] = h;
    const double x = sx[c];
    xHI[c] = x;
    xHII[c] = sz ? sz[c] : __dsub_rn(1.0, x);
    const double v = __dmul_rn(h, x);
    if (PAIR) {
      const F2 p = f2_from_double(v);
      ((float2*)nhi)[c] = make_float2(p.hi, p.lo);
    } else {
      ((double*)nhi)[c] = v;
    }
  }
  commit_finish(ctl);
}

// The same commit two cells at a time (16-byte accesses), for 16-byte
// aligned arrays of an even length.
template <bool PAIR>
__global__ void commit_state2_kernel(long long n2, unsigned long long* __restrict__ ctl, const double2* __restrict__ sn,
                                     const double2* __restrict__ sx, const double2* __restrict__ sz,
                                     double2* __restrict__ nH, double2* __restrict__ xHI, double2* __restrict__ xHII,
                                     void* __restrict__ nhi) {
  const bool ok = commit_verdict(ctl);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; ok && i < n2;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 h = sn ? sn[i] : nH[i];
    if (sn) nH[i] = h;
    const double2 x = sx[i];
    xHI[i] = x;
    xHII[i] = sz ? sz[i] : make_double2(__dsub_rn(1.0, x.x), __dsub_rn(1.0, x.y));
    const double v0 = __dmul_rn(h.x, x.x), v1 = __dmul_rn(h.y, x.y);
    if (PAIR) {
      const F2 p0 = f2_from_double(v0), p1 = f2_from_double(v1);
      ((float4*)nhi)[i] = make_float4(p0.hi, p0.lo, p1.hi, p1.lo);
    } else {
      ((double2*)nhi)[i] = make_double2(v0, v1);
    }
  }
  commit_finish(ctl);
}

// Commit of a state uploaded straight into the grid's alternate buffers
// (rt_set_state_async from host memory without n_H; the host has already
// made x and z the grid's arrays).  Every block checks its cells' x_HI and
// writes their n_HI = n_H x_HI (and x_HII = 1 - x_HI when none was uploaded)
// as if the state passed; the block that finishes last (CTL_COMMIT_DONE)
// takes the verdict.  A rejected state is undone by that block -- the
// previous state copied into x and z and n_HI recomputed from it, so the
// grid ends as it was -- and latched in ctl[CTL_SET_ERR].  Either way it
// points the grid's device descriptor at x and z and sets the check words
// back to ~0.
template <bool PAIR>
__global__ void check_refresh_kernel(long long n, unsigned long long* __restrict__ ctl, const double* __restrict__ nH,
                                     double* __restrict__ x, double* __restrict__ z, int z_given,
                                     const double* __restrict__ x_old, const double* __restrict__ z_old,
                                     void* __restrict__ nhi, InstDev* __restrict__ inst) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const double xv = x[c];
    if (!(xv >= 0.0 && xv <= 1.0)) atomicMin(&ctl[CTL_CHECK_X], (unsigned long long)c);
    if (!z_given) z[c] = __dsub_rn(1.0, xv);
    const double v = __dmul_rn(nH[c], xv);
    if (PAIR) {
      const F2 p = f2_from_double(v);
      ((float2*)nhi)[c] = make_float2(p.hi, p.lo);
    } else {
      ((double*)nhi)[c] = v;
    }
  }
  __shared__ int last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&ctl[CTL_COMMIT_DONE], 1ULL) == (unsigned long long)gridDim.x - 1ULL;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const unsigned long long bx = ctl[CTL_CHECK_X];
  if (bx != ~0ULL) {
    if (threadIdx.x == 0 && atomicCAS(&ctl[CTL_SET_ERR], 0ULL, (unsigned long long)RT_ERR_INVALID_ARG) == 0ULL) {
      ctl[CTL_SET_BADN] = ~0ULL;
      ctl[CTL_SET_BADX] = bx;
    }
    for (long long c = threadIdx.x; c < n; c += blockDim.x) {
      const double xv = x_old[c];
      x[c] = xv;
      z[c] = z_old[c];
      const double v = __dmul_rn(nH[c], xv);
      if (PAIR) {
        const F2 p = f2_from_double(v);
        ((float2*)nhi)[c] = make_float2(p.hi, p.lo);
      } else {
        ((double*)nhi)[c] = v;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    inst->xHI = x;
    inst->xHII = z;
    ctl[CTL_CHECK_N] = ~0ULL;
    ctl[CTL_CHECK_X] = ~0ULL;
    ctl[CTL_COMMIT_DONE] = 0ULL;
  }
}

// Adaptive RT timestep (Sec. 3.4), step 1, Eq. "dtelec": per cell
// eps / |k_ph + n_e alpha_B| (C_H = 0, n_e = n_H (1 - x_HI)) where the cell's
// optical depth sdx n_HI exceeds tau_front, else dt_max; never above dt_max.
// The front test is FP64 (a cell's side of the threshold must not depend on
// rounding); the value is FP32 (a timestep needs no more), in units of
// dt_max when dt_max is finite (so cells outside the front hold exactly 1).
template <typename KT>
__global__ void cell_timestep_kernel(long long n, const double* __restrict__ nH, const double* __restrict__ xHI,
                                     const KT* __restrict__ K, double sdx, double tau_front, float eps, float alpha,
                                     float dt_max, float unit, float* __restrict__ dtc) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const double nh64 = nH[c], x64 = xHI[c];
    const float nh = (float)nh64, x = (float)x64;
    const float rate = fabsf((float)K[c] + nh * (1.0f - x) * alpha);
    float dt = dt_max;
    if (sdx * nh64 * x64 > tau_front && rate > 0.0f) dt = fminf(dt_max, eps / rate);
    dtc[c] = dt == dt_max ? dt_max / unit : dt / unit;
  }
}

// Steps 2-3: the 3^3 Gaussian (exp(-|d|^2/2), renormalised over neighbours
// inside the grid) of the per-cell timestep, and its minimum over the grid
// (atomicMin on the bit patterns, which order like the positive floats).
__global__ void smooth_min_kernel(const float* __restrict__ dtc, int nx, int ny, int nz, unsigned int* __restrict__ out) {
  const float w1 = 0.60653066f, w2 = 0.36787944f, w3 = 0.22313016f;  // e^-1/2, e^-1, e^-3/2
  const long long n = (long long)nx * ny * nz;
  float best = __int_as_float(0x7f800000);
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((long long)nx * ny));
    float acc = 0.0f, ws = 0.0f;
    for (int dz = -1; dz <= 1; ++dz) {
      const int kk = k + dz;
      if (kk < 0 || kk >= nz) continue;
      for (int dy = -1; dy <= 1; ++dy) {
        const int jj = j + dy;
        if (jj < 0 || jj >= ny) continue;
        for (int dxo = -1; dxo <= 1; ++dxo) {
          const int ii = i + dxo;
          if (ii < 0 || ii >= nx) continue;
          const int d2 = dxo * dxo + dy * dy + dz * dz;
          const float w = d2 == 0 ? 1.0f : (d2 == 1 ? w1 : (d2 == 2 ? w2 : w3));
          acc = fmaf(w, dtc[ii + (long long)nx * (jj + (long long)ny * kk)], acc);
          ws += w;
        }
      }
    }
    best = fminf(best, acc / ws);
  }
  for (int o = 16; o > 0; o >>= 1) best = fminf(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) atomicMin(out, __float_as_uint(best));
}

cudaError_t launch_timestep(long long n, int nx, int ny, int nz, const double* nH, const double* xHI, const void* K,
                            int fp64_rates, double sdx, double tau_front, float eps, float alpha, float dt_max,
                            float unit, float* dtc, unsigned int* out, cudaStream_t st) {
  const int block = 256;
  long long g = (n + block - 1) / block;
  if (g > 152 * 8) g = 152 * 8;
  if (g < 1) g = 1;
  if (fp64_rates)
    cell_timestep_kernel<double><<<(int)g, block, 0, st>>>(n, nH, xHI, (const double*)K, sdx, tau_front, eps, alpha,
                                                          dt_max, unit, dtc);
  else
    cell_timestep_kernel<float><<<(int)g, block, 0, st>>>(n, nH, xHI, (const float*)K, sdx, tau_front, eps, alpha,
                                                         dt_max, unit, dtc);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  smooth_min_kernel<<<(int)g, block, 0, st>>>(dtc, nx, ny, nz, out);
  return cudaGetLastError();
}

// h alpha_B and h as FP32 pairs (host side), for the mixed update kernels
static float4 step_pairs(double h, double alpha) {
  const double ha = h * alpha;
  const float a_hi = (float)ha, h_hi = (float)h;
  return make_float4(a_hi, (float)(ha - (double)a_hi), h_hi, (float)(h - (double)h_hi));
}

static int grid_for(long long n, int block) {
  long long g = (n + block - 1) / block;
  if (g > 152 * 32) g = 152 * 32;
  if (g < 1) g = 1;
  return (int)g;
}

cudaError_t launch_chem(int precision, long long ncell, const double* nH, double* xHI, double* xHII,
                        const void* K, void* nhi, double h, int nsub, double alpha, cudaStream_t st) {
  const int block = 256, grid = grid_for(ncell, block);
  if (precision == RT_FP64)
    chem_kernel<double, double><<<grid, block, 0, st>>>(ncell, nH, xHI, xHII, (const double*)K,
                                                         (double*)nhi, h, nsub, alpha);
  else
    chem_mixed_kernel<<<grid, block, 0, st>>>(ncell, nH, xHI, xHII, (const float*)K, (float2*)nhi,
                                              step_pairs(h, alpha), nsub);
  return cudaGetLastError();
}

cudaError_t launch_refresh(int precision, long long ncell, const double* nH, const double* xHI,
                           void* nhi, cudaStream_t st) {
  const int block = 256, grid = grid_for(ncell, block);
  if (precision == RT_FP64)
    refresh_nhi_kernel<double><<<grid, block, 0, st>>>(ncell, nH, xHI, (double*)nhi);
  else
    refresh_nhi_pair_kernel<<<grid, block, 0, st>>>(ncell, nH, xHI, (float2*)nhi);
  return cudaGetLastError();
}

cudaError_t launch_pair(long long n, const double* src, void* dst, cudaStream_t st) {
  const int block = 256, grid = grid_for(n, block);
  pair_kernel<<<grid, block, 0, st>>>(n, src, (float2*)dst);
  return cudaGetLastError();
}

cudaError_t launch_check_density(long long n, const double* a, unsigned long long* bad, cudaStream_t st) {
  const int block = 256, grid = grid_for(n, block);
  check_density_kernel<<<grid, block, 0, st>>>(n, a, bad);
  return cudaGetLastError();
}

// Adds delta to one device word (the trace self-test's phantom package).
// Step 2 of a trace in one launch: k_ph and Gamma (two arrays of nbytes
// each, 16-byte aligned) and the budget words (acc, cnt) to zero.
__global__ void zero_fields_kernel(uint4* __restrict__ a, uint4* __restrict__ b, size_t n16, size_t nbytes,
                                   unsigned long long* __restrict__ acc, int nacc, unsigned long long* __restrict__ cnt,
                                   int ncnt) {
  const uint4 z = make_uint4(0u, 0u, 0u, 0u);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n16; i += (size_t)gridDim.x * blockDim.x) {
    a[i] = z;
    b[i] = z;
  }
  if (blockIdx.x == 0) {
    for (size_t t = 16 * n16 + threadIdx.x; t < nbytes; t += blockDim.x) {
      ((unsigned char*)a)[t] = 0;
      ((unsigned char*)b)[t] = 0;
    }
    for (int t = threadIdx.x; t < nacc; t += blockDim.x) acc[t] = 0ULL;
    for (int t = threadIdx.x; t < ncnt; t += blockDim.x) cnt[t] = 0ULL;
  }
}

cudaError_t launch_zero_fields(void* a, void* b, size_t nbytes, void* acc, int nacc, void* cnt, int ncnt,
                               cudaStream_t st) {
  if (((uintptr_t)a & 15u) || ((uintptr_t)b & 15u)) return cudaErrorInvalidValue;
  const size_t n16 = nbytes / 16;
  long long blocks = (long long)((n16 + 255) / 256);
  if (blocks > 152 * 4) blocks = 152 * 4;
  if (blocks < 1) blocks = 1;
  zero_fields_kernel<<<(int)blocks, 256, 0, st>>>((uint4*)a, (uint4*)b, n16, nbytes, (unsigned long long*)acc, nacc,
                                                  (unsigned long long*)cnt, ncnt);
  return cudaGetLastError();
}

__global__ void add_word_kernel(unsigned long long* w, unsigned long long delta) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *w += delta;
}

cudaError_t launch_add_word(unsigned long long* w, unsigned long long delta, cudaStream_t st) {
  add_word_kernel<<<1, 32, 0, st>>>(w, delta);
  return cudaGetLastError();
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

cudaError_t launch_check_state(long long n, const double* nH, const double* x, unsigned long long* bad,
                               cudaStream_t st) {
  const int block = 256;
  if (n % 2 == 0 && aligned16(nH) && aligned16(x))
    check_state2_kernel<<<grid_for(n / 2, block), block, 0, st>>>(n / 2, (const double2*)nH, (const double2*)x, bad);
  else
    check_state_kernel<<<grid_for(n, block), block, 0, st>>>(n, nH, x, bad);
  return cudaGetLastError();
}

cudaError_t launch_commit_state(int precision, long long n, unsigned long long* ctl, const double* sn,
                               const double* sx, const double* sz, double* nH, double* xHI, double* xHII, void* nhi,
                               cudaStream_t st) {
  const int block = 256;
  if (n % 2 == 0 && aligned16(sn) && aligned16(sx) && aligned16(sz) && aligned16(nH) && aligned16(xHI) &&
      aligned16(xHII) && aligned16(nhi)) {
    const long long n2 = n / 2;
    const int grid = grid_for(n2, block);
    if (precision == RT_FP64)
      commit_state2_kernel<false><<<grid, block, 0, st>>>(n2, ctl, (const double2*)sn, (const double2*)sx,
                                                          (const double2*)sz, (double2*)nH, (double2*)xHI,
                                                          (double2*)xHII, nhi);
    else
      commit_state2_kernel<true><<<grid, block, 0, st>>>(n2, ctl, (const double2*)sn, (const double2*)sx,
                                                         (const double2*)sz, (double2*)nH, (double2*)xHI,
                                                         (double2*)xHII, nhi);
    return cudaGetLastError();
  }
  const int grid = grid_for(n, block);
  if (precision == RT_FP64)
    commit_state_kernel<false><<<grid, block, 0, st>>>(n, ctl, sn, sx, sz, nH, xHI, xHII, nhi);
  else
    commit_state_kernel<true><<<grid, block, 0, st>>>(n, ctl, sn, sx, sz, nH, xHI, xHII, nhi);
  return cudaGetLastError();
}

cudaError_t launch_check_refresh(int precision, long long n, unsigned long long* ctl, const double* nH, double* x,
                                 double* z, int z_given, const double* x_old, const double* z_old, void* nhi,
                                 InstDev* inst, cudaStream_t st) {
  const int block = 256, grid = grid_for(n, block);
  if (precision == RT_FP64)
    check_refresh_kernel<false><<<grid, block, 0, st>>>(n, ctl, nH, x, z, z_given, x_old, z_old, nhi, inst);
  else
    check_refresh_kernel<true><<<grid, block, 0, st>>>(n, ctl, nH, x, z, z_given, x_old, z_old, nhi, inst);
  return cudaGetLastError();
}

cudaError_t launch_complement(long long n, const double* x, double* out, cudaStream_t st) {
  const int block = 256, grid = grid_for(n, block);
  complement_kernel<<<grid, block, 0, st>>>(n, x, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Batched forms: one launch for every grid of a batch.  blockIdx.y selects the
// grid (its descriptor in `inst`), blocks of a row stride over its cells.
// ---------------------------------------------------------------------------

// Step 2 for every grid: zero k_ph, Gamma (element size esz), the budget
// sums and the counters.
__global__ void batch_zero_kernel(const InstDev* __restrict__ inst, int esz) {
  const InstDev I = inst[blockIdx.y];
  const long long n = (long long)I.nx * I.ny * I.nz;
  const long long words = n * esz / 4;
  unsigned int* K = (unsigned int*)I.K;
  unsigned int* G = (unsigned int*)I.G;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < words;
       c += (long long)gridDim.x * blockDim.x) {
    K[c] = 0u;
    G[c] = 0u;
  }
  for (int t = 0; t < 2; ++t) {  // helium photon types, where the grid has them
    if (!I.Khe[t]) continue;
    unsigned int* Kt = (unsigned int*)I.Khe[t];
    unsigned int* Gt = (unsigned int*)I.Ghe[t];
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < words;
         c += (long long)gridDim.x * blockDim.x) {
      Kt[c] = 0u;
      Gt[c] = 0u;
    }
  }
  if (blockIdx.x == 0) {
    for (int i = threadIdx.x; i < 8; i += blockDim.x) I.acc[i] = 0.0;
    for (int i = threadIdx.x; i < kCntWords; i += blockDim.x) I.cnt[i] = 0ULL;
  }
}

template <bool MIXED>
__global__ void batch_chem_kernel(const InstDev* __restrict__ inst, double h, int nsub, double alpha, float4 hh) {
  const InstDev I = inst[blockIdx.y];
  const F2 ha = {hh.x, hh.y}, h2 = {hh.z, hh.w};
  const long long n = (long long)I.nx * I.ny * I.nz;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    double x = I.xHI[c], z = I.xHII[c];
    if (MIXED) {
      const float kc = ((const float*)I.K)[c];
      if (kc == 0.0f && is_neutral(x, z)) continue;
      const F2 nx = chem_cell_mixed(x, z, I.nH[c], kc, ha, h2, nsub);
      ((double*)I.xHI)[c] = x;
      I.xHII[c] = z;
      ((float2*)I.nhi)[c] = make_float2(nx.hi, nx.lo);
    } else {
      const double kc = ((const double*)I.K)[c];
      if (kc == 0.0 && z == 0.0 && x == 1.0) continue;
      const double nh = I.nH[c];
      chem_cell_fp64(x, z, nh, kc, h, nsub, alpha);
      ((double*)I.xHI)[c] = x;
      I.xHII[c] = z;
      ((double*)I.nhi)[c] = __dmul_rn(nh, x);
    }
  }
}

cudaError_t launch_batch_zero(const InstDev* inst, int ninst, int precision, long long max_cells, cudaStream_t st) {
  if (ninst <= 0) return cudaSuccess;
  const int esz = precision == RT_FP64 ? 8 : 4;
  long long bx = (max_cells * esz / 4 + 255) / 256;
  if (bx > 64) bx = 64;
  if (bx < 1) bx = 1;
  batch_zero_kernel<<<dim3((unsigned)bx, (unsigned)ninst), 256, 0, st>>>(inst, esz);
  return cudaGetLastError();
}

cudaError_t launch_batch_chem(const InstDev* inst, int ninst, int precision, long long max_cells, double h,
                              int nsub, double alpha, cudaStream_t st) {
  if (ninst <= 0) return cudaSuccess;
  // blocks per grid for ~4096 cells each (up to 1024): a grid's cells are
  // spread over blocks in proportion to its size, so the largest grids of a
  // batch do not finish last on a few blocks; the blocks a smaller grid does
  // not need return at once.  (64 blocks per grid took 4.0 vs 2.5 ms on the
  // 64-grid batch.)
  long long bx = (max_cells + 4095) / 4096;
  if (bx > 1024) bx = 1024;
  if (bx < 1) bx = 1;
  if (precision == RT_FP64)
    batch_chem_kernel<false><<<dim3((unsigned)bx, (unsigned)ninst), 256, 0, st>>>(inst, h, nsub, alpha,
                                                                                   step_pairs(h, alpha));
  else
    batch_chem_kernel<true><<<dim3((unsigned)bx, (unsigned)ninst), 256, 0, st>>>(inst, h, nsub, alpha,
                                                                                  step_pairs(h, alpha));
  return cudaGetLastError();
}

// src_dtype / dst_dtype: RT_DTYPE_F64 or RT_DTYPE_F32; dst = src * scale
// (the product in FP64)
cudaError_t launch_convert(long long n, const void* src, int src_dtype, void* dst, int dst_dtype,
                           cudaStream_t st, double scale) {
  const int block = 256, grid = grid_for(n, block);
  if (src_dtype == RT_DTYPE_F64 && dst_dtype == RT_DTYPE_F64)
    convert_kernel<double, double><<<grid, block, 0, st>>>(n, (const double*)src, (double*)dst, scale);
  else if (src_dtype == RT_DTYPE_F64 && dst_dtype == RT_DTYPE_F32)
    convert_kernel<double, float><<<grid, block, 0, st>>>(n, (const double*)src, (float*)dst, scale);
  else if (src_dtype == RT_DTYPE_F32 && dst_dtype == RT_DTYPE_F64)
    convert_kernel<float, double><<<grid, block, 0, st>>>(n, (const float*)src, (double*)dst, scale);
  else
    convert_kernel<float, float><<<grid, block, 0, st>>>(n, (const float*)src, (float*)dst, scale);
  return cudaGetLastError();
}

}  // namespace rtg
