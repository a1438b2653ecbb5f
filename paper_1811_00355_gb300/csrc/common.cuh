// Device-side building blocks shared by the kernels of the library:
// complex arithmetic, the block-major structure-of-arrays field layout, the
// Wilson spin projectors in the chiral basis, SU(3) link reconstruction and
// the packed Hermitian 6x6 clover product.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "kernels.h"

namespace ddamg {

// ---------------------------------------------------------------------------
// complex numbers
// ---------------------------------------------------------------------------
template <class R>
struct cpx {
  R re, im;
};

__host__ __device__ __forceinline__ float fma_r(float a, float b, float c) { return fmaf(a, b, c); }
__host__ __device__ __forceinline__ double fma_r(double a, double b, double c) { return ::fma(a, b, c); }

template <class R> __host__ __device__ __forceinline__ cpx<R> mk(R a, R b) { return {a, b}; }
template <class R> __host__ __device__ __forceinline__ cpx<R> operator+(cpx<R> a, cpx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <class R> __host__ __device__ __forceinline__ cpx<R> operator-(cpx<R> a, cpx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <class R> __host__ __device__ __forceinline__ cpx<R> operator-(cpx<R> a) { return {-a.re, -a.im}; }
template <class R> __host__ __device__ __forceinline__ cpx<R> operator*(cpx<R> a, cpx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <class R> __host__ __device__ __forceinline__ cpx<R> operator*(R s, cpx<R> a) { return {s * a.re, s * a.im}; }
template <class R> __host__ __device__ __forceinline__ cpx<R> conj(cpx<R> a) { return {a.re, -a.im}; }
// a * b with a conjugated
template <class R> __host__ __device__ __forceinline__ cpx<R> cmulc(cpx<R> a, cpx<R> b) {
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
// i * a and -i * a
template <class R> __host__ __device__ __forceinline__ cpx<R> ti(cpx<R> a) { return {-a.im, a.re}; }
template <class R> __host__ __device__ __forceinline__ cpx<R> tmi(cpx<R> a) { return {a.im, -a.re}; }
// acc += a * b (fused)
template <class R> __host__ __device__ __forceinline__ void fma(cpx<R>& acc, cpx<R> a, cpx<R> b) {
  acc.re = fma_r(a.re, b.re, fma_r(-a.im, b.im, acc.re));
  acc.im = fma_r(a.re, b.im, fma_r(a.im, b.re, acc.im));
}
// acc += conj(a) * b
template <class R> __host__ __device__ __forceinline__ void fmac(cpx<R>& acc, cpx<R> a, cpx<R> b) {
  acc.re = fma_r(a.re, b.re, fma_r(a.im, b.im, acc.re));
  acc.im = fma_r(a.re, b.im, fma_r(-a.im, b.re, acc.im));
}
template <class R> __host__ __device__ __forceinline__ R norm2(cpx<R> a) { return a.re * a.re + a.im * a.im; }

// ---------------------------------------------------------------------------
// field layout: block-major structure of arrays of 16-byte units
//   a field of NR reals per site is stored as [block][unit][site in block],
//   unit = 16 bytes (float4 or double2); device site d = block*Vb + q with
//   q = parity*(Vb/2) + (local lexicographic index >> 1).
//   Several right-hand sides follow one another (stride V*NR reals).
// ---------------------------------------------------------------------------
template <class R> struct U16;
template <> struct U16<float> { using T = float4; static constexpr int N = 4; };
template <> struct U16<double> { using T = double2; static constexpr int N = 2; };

template <class R, int NR>
struct Layout {
  static constexpr int PER = U16<R>::N;     // reals per unit
  static constexpr int NU = NR / PER;       // units per site
  static_assert(NR % PER == 0, "field width must be a whole number of units");
  // offset (in units) of unit 0 of site d; unit u sits u*Vb units further
  __device__ __forceinline__ static size_t base(int d, int Vb) {
    int B = d / Vb;
    int q = d - B * Vb;
    return (size_t)B * NU * Vb + q;
  }
};

template <class R>
__device__ __forceinline__ void st_unit(R* p, size_t off, const R* v);
template <>
__device__ __forceinline__ void st_unit<float>(float* p, size_t off, const float* v) {
  reinterpret_cast<float4*>(p)[off] = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ void st_unit<double>(double* p, size_t off, const double* v) {
  reinterpret_cast<double2*>(p)[off] = make_double2(v[0], v[1]);
}
template <class R>
__device__ __forceinline__ void ld_unit(const R* p, size_t off, R* v);
template <>
__device__ __forceinline__ void ld_unit<float>(const float* p, size_t off, float* v) {
  float4 t = __ldg(reinterpret_cast<const float4*>(p) + off);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
template <>
__device__ __forceinline__ void ld_unit<double>(const double* p, size_t off, double* v) {
  double2 t = __ldg(reinterpret_cast<const double2*>(p) + off);
  v[0] = t.x; v[1] = t.y;
}
// plain (non-__ldg) load for data written earlier in the same kernel
template <class R>
__device__ __forceinline__ void ld_unit_cg(const R* p, size_t off, R* v);
template <>
__device__ __forceinline__ void ld_unit_cg<float>(const float* p, size_t off, float* v) {
  float4 t = __ldcg(reinterpret_cast<const float4*>(p) + off);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
template <>
__device__ __forceinline__ void ld_unit_cg<double>(const double* p, size_t off, double* v) {
  double2 t = __ldcg(reinterpret_cast<const double2*>(p) + off);
  v[0] = t.x; v[1] = t.y;
}

// load / store NR reals of site d
template <class R, int NR>
__device__ __forceinline__ void load_site(const R* __restrict__ f, int d, int Vb, R* v) {
  using LY = Layout<R, NR>;
  size_t b = LY::base(d, Vb);
#pragma unroll
  for (int u = 0; u < LY::NU; ++u) ld_unit<R>(f, b + (size_t)u * Vb, v + u * LY::PER);
}
template <class R, int NR>
__device__ __forceinline__ void load_site_cg(const R* f, int d, int Vb, R* v) {
  using LY = Layout<R, NR>;
  size_t b = LY::base(d, Vb);
#pragma unroll
  for (int u = 0; u < LY::NU; ++u) ld_unit_cg<R>(f, b + (size_t)u * Vb, v + u * LY::PER);
}
template <class R, int NR>
__device__ __forceinline__ void store_site(R* __restrict__ f, int d, int Vb, const R* v) {
  using LY = Layout<R, NR>;
  size_t b = LY::base(d, Vb);
#pragma unroll
  for (int u = 0; u < LY::NU; ++u) st_unit<R>(f, b + (size_t)u * Vb, v + u * LY::PER);
}
// load the units [u0, u0 + n) of site d
template <class R, int NR>
__device__ __forceinline__ void load_units(const R* __restrict__ f, int d, int Vb, int u0, int n, R* v) {
  using LY = Layout<R, NR>;
  size_t b = LY::base(d, Vb) + (size_t)u0 * Vb;
  for (int u = 0; u < n; ++u) ld_unit<R>(f, b + (size_t)u * Vb, v + u * LY::PER);
}

// widths in reals
constexpr int SPINOR_NR = 24;   // 4 spins x 3 colours complex
constexpr int LINK_NR = 12;     // two rows of an SU(3) matrix
constexpr int GAUGE_NR = 48;    // 4 links per site
constexpr int CLOVER_NR = 72;   // two packed Hermitian 6x6 blocks

template <class R>
struct Spinor {
  cpx<R> c[12];   // index spin*3 + colour
};

template <class R>
__device__ __forceinline__ void load_spinor(const R* f, int d, int Vb, Spinor<R>& s) {
  load_site<R, SPINOR_NR>(f, d, Vb, reinterpret_cast<R*>(s.c));
}
template <class R>
__device__ __forceinline__ void load_spinor_cg(const R* f, int d, int Vb, Spinor<R>& s) {
  load_site_cg<R, SPINOR_NR>(f, d, Vb, reinterpret_cast<R*>(s.c));
}
template <class R>
__device__ __forceinline__ void store_spinor(R* f, int d, int Vb, const Spinor<R>& s) {
  store_site<R, SPINOR_NR>(f, d, Vb, reinterpret_cast<const R*>(s.c));
}

// ---------------------------------------------------------------------------
// SU(3): third row rebuilt as conj(row0 x row1)
// ---------------------------------------------------------------------------
template <class R>
struct Link {
  cpx<R> m[3][3];
};

template <class R>
__device__ __forceinline__ void complete_link(Link<R>& U) {
  U.m[2][0] = conj(U.m[0][1] * U.m[1][2] - U.m[0][2] * U.m[1][1]);
  U.m[2][1] = conj(U.m[0][2] * U.m[1][0] - U.m[0][0] * U.m[1][2]);
  U.m[2][2] = conj(U.m[0][0] * U.m[1][1] - U.m[0][1] * U.m[1][0]);
}

template <class R>
__device__ __forceinline__ void load_link(const R* __restrict__ g, int d, int Vb, int mu, Link<R>& U) {
  using LY = Layout<R, GAUGE_NR>;
  constexpr int NUL = LINK_NR / LY::PER;   // units per link
  R v[LINK_NR];
  size_t b = LY::base(d, Vb) + (size_t)(mu * NUL) * Vb;
#pragma unroll
  for (int u = 0; u < NUL; ++u) ld_unit<R>(g, b + (size_t)u * Vb, v + u * LY::PER);
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    U.m[k / 3][k % 3] = mk(v[2 * k], v[2 * k + 1]);
  }
  complete_link(U);
}

// y = U h (both spin rows of a half spinor h[2][3])
template <class R>
__device__ __forceinline__ void su3_mul(const Link<R>& U, const cpx<R> h[2][3], cpx<R> y[2][3]) {
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cpx<R> acc = U.m[a][0] * h[s][0];
      fma(acc, U.m[a][1], h[s][1]);
      fma(acc, U.m[a][2], h[s][2]);
      y[s][a] = acc;
    }
}
// y = U^H h
template <class R>
__device__ __forceinline__ void su3_mul_dag(const Link<R>& U, const cpx<R> h[2][3], cpx<R> y[2][3]) {
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cpx<R> acc = cmulc(U.m[0][a], h[s][0]);
      fmac(acc, U.m[1][a], h[s][1]);
      fmac(acc, U.m[2][a], h[s][2]);
      y[s][a] = acc;
    }
}

// ---------------------------------------------------------------------------
// Wilson projectors in the chiral basis.  With g_mu = [[0, B],[B^H, 0]]:
//   (1 - g_mu) psi = [h; -B^H h],  h = psi_up - B psi_dn
//   (1 + g_mu) psi = [h;  B^H h],  h = psi_up + B psi_dn
// B_x = -i s1, B_y = -i s2, B_z = -i s3, B_t = 1.
// project<MU, SIGN>: SIGN = -1 for (1 - g_mu), +1 for (1 + g_mu).
// ---------------------------------------------------------------------------
template <int MU, int SIGN, class R>
__device__ __forceinline__ void project(const Spinor<R>& p, cpx<R> h[2][3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    cpx<R> s0 = p.c[0 * 3 + a], s1 = p.c[1 * 3 + a], s2 = p.c[2 * 3 + a], s3 = p.c[3 * 3 + a];
    if (MU == 0) {         // B psi_dn = (-i s3, -i s2)
      if (SIGN < 0) { h[0][a] = s0 + ti(s3); h[1][a] = s1 + ti(s2); }
      else          { h[0][a] = s0 + tmi(s3); h[1][a] = s1 + tmi(s2); }
    } else if (MU == 1) {  // B psi_dn = (-s3, s2)
      if (SIGN < 0) { h[0][a] = s0 + s3; h[1][a] = s1 - s2; }
      else          { h[0][a] = s0 - s3; h[1][a] = s1 + s2; }
    } else if (MU == 2) {  // B psi_dn = (-i s2, i s3)
      if (SIGN < 0) { h[0][a] = s0 + ti(s2); h[1][a] = s1 + tmi(s3); }
      else          { h[0][a] = s0 + tmi(s2); h[1][a] = s1 + ti(s3); }
    } else {               // B psi_dn = (s2, s3)
      if (SIGN < 0) { h[0][a] = s0 - s2; h[1][a] = s1 - s3; }
      else          { h[0][a] = s0 + s2; h[1][a] = s1 + s3; }
    }
  }
}

// acc += [y; -+B^H y] (reconstruction of the lower spins), scaled by sc
template <int MU, int SIGN, class R>
__device__ __forceinline__ void accumulate(Spinor<R>& acc, const cpx<R> y[2][3], R sc) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    cpx<R> y0 = sc * y[0][a], y1 = sc * y[1][a];
    acc.c[0 * 3 + a] = acc.c[0 * 3 + a] + y0;
    acc.c[1 * 3 + a] = acc.c[1 * 3 + a] + y1;
    cpx<R> l2, l3;
    // B^H: x: (i s1) y = (i y1, i y0); y: (i s2) y = (y1, -y0);
    //      z: (i s3) y = (i y0, -i y1); t: y
    if (MU == 0)      { l2 = ti(y1);  l3 = ti(y0); }
    else if (MU == 1) { l2 = y1;      l3 = -y0; }
    else if (MU == 2) { l2 = ti(y0);  l3 = tmi(y1); }
    else              { l2 = y0;      l3 = y1; }
    if (SIGN < 0) { l2 = -l2; l3 = -l3; }
    acc.c[2 * 3 + a] = acc.c[2 * 3 + a] + l2;
    acc.c[3 * 3 + a] = acc.c[3 * 3 + a] + l3;
  }
}

// ---------------------------------------------------------------------------
// packed Hermitian 6x6 (36 reals: 6 real diagonal, 15 upper complex row-major)
// y = H v
// ---------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ void herm6(const R* P, const cpx<R>* v, cpx<R>* y) {
#pragma unroll
  for (int i = 0; i < 6; ++i) y[i] = P[i] * v[i];
  int k = 0;
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = i + 1; j < 6; ++j) {
      cpx<R> a = mk(P[6 + 2 * k], P[7 + 2 * k]);
      fma(y[i], a, v[j]);
      fmac(y[j], a, v[i]);
      ++k;
    }
}

// y = A(site) v with the two chiral blocks of a packed clover field
template <class R>
__device__ __forceinline__ void clover_mul(const R* __restrict__ clov, int d, int Vb, const Spinor<R>& v, Spinor<R>& y) {
  using LY = Layout<R, CLOVER_NR>;
  constexpr int NUB = 36 / LY::PER;   // units per chiral block
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    R P[36];
    load_units<R, CLOVER_NR>(clov, d, Vb, s * NUB, NUB, P);
    herm6<R>(P, v.c + 6 * s, y.c + 6 * s);
  }
}

// ---------------------------------------------------------------------------
// bulk asynchronous copies (TMA, untiled) global -> shared, completed on an
// mbarrier; addresses 16-byte aligned, sizes multiples of 16 bytes
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait on phase `parity`; false after `limit` unsuccessful polls
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, long long limit) {
  for (long long n = 0; n < limit; ++n)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
constexpr long long MBAR_POLL_LIMIT = 1ll << 22;

// neighbour table entries: device index with bit 31 set when the hop carries
// the antiperiodic sign
constexpr uint32_t NEG_BIT = 0x80000000u;

// ---------------------------------------------------------------------------
// Wilson hopping term of one direction at device site d (neighbours from the
// global table, fields in global memory):
//   acc += (1 - g_mu) U_mu(x) x(x+mu) + (1 + g_mu) U_mu(x-mu)^H x(x-mu)
// ---------------------------------------------------------------------------
template <int MU, class R>
__device__ __forceinline__ void hop_dir(const Geom& g, const R* __restrict__ x,
                                        const R* __restrict__ gauge, int d, Spinor<R>& acc) {
  cpx<R> h[2][3], y[2][3];
  Spinor<R> nb;
  {  // forward: (1 - g_mu) U_mu(x) x(x+mu)
    uint32_t e = __ldg(g.nbr + (size_t)(2 * MU) * g.V + d);
    int n = (int)(e & ~NEG_BIT);
    R sc = (e & NEG_BIT) ? R(-1) : R(1);
    load_spinor<R>(x, n, g.Vb, nb);
    project<MU, -1>(nb, h);
    Link<R> U;
    load_link<R>(gauge, d, g.Vb, MU, U);
    su3_mul(U, h, y);
    accumulate<MU, -1>(acc, y, sc);
  }
  {  // backward: (1 + g_mu) U_mu(x-mu)^H x(x-mu)
    uint32_t e = __ldg(g.nbr + (size_t)(2 * MU + 1) * g.V + d);
    int n = (int)(e & ~NEG_BIT);
    R sc = (e & NEG_BIT) ? R(-1) : R(1);
    load_spinor<R>(x, n, g.Vb, nb);
    project<MU, +1>(nb, h);
    Link<R> U;
    load_link<R>(gauge, n, g.Vb, MU, U);
    su3_mul_dag(U, h, y);
    accumulate<MU, +1>(acc, y, sc);
  }
}


}  // namespace ddamg
