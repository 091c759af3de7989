// Point updates of the complex 5-point Helmholtz operator with PML stretching (eq. 3 in
// stretched coordinates, multiplied through by s_x s_y: the complex-symmetric form).
#pragma once

#include "helm_internal.cuh"

namespace helm {

// General point update: -(1/h^2)[s_y(j)((uE-uC)/s_x(i+1/2) - (uC-uW)/s_x(i-1/2))
//                               + s_x(i)((uN-uC)/s_y(j+1/2) - (uC-uS)/s_y(j-1/2))] - s_x s_y k^2 uC
template <typename R>
__device__ __forceinline__ C<R> stencil_point(C<R> uC, C<R> uE, C<R> uW, C<R> uN, C<R> uS, C<R> sxi, C<R> ixm,
                                              C<R> ixp, C<R> syj, C<R> iym, C<R> iyp, R k2, R inv_h2) {
  C<R> fx = csub(cmul(csub(uE, uC), ixp), cmul(csub(uC, uW), ixm));
  C<R> fy = csub(cmul(csub(uN, uC), iyp), cmul(csub(uC, uS), iym));
  C<R> acc = cadd(cmul(syj, fx), cmul(sxi, fy));
  C<R> sxy = cmul(sxi, syj);
  C<R> diag = cmul(sxy, uC);
  C<R> r;
  r.x = -acc.x * inv_h2 - k2 * diag.x;
  r.y = -acc.y * inv_h2 - k2 * diag.y;
  return r;
}

template <typename R>
__device__ __forceinline__ bool unit_c(C<R> v) { return v.x == (R)1 && v.y == (R)0; }

// The point update where every stretch factor is exactly 1 + 0i (outside the PML): the general
// form above reduces exactly to this, evaluated in the same order.
template <typename R>
__device__ __forceinline__ C<R> stencil_point_unit(C<R> uC, C<R> uE, C<R> uW, C<R> uN, C<R> uS, R k2, R inv_h2) {
  C<R> r;
  r.x = -(((uE.x - uC.x) - (uC.x - uW.x)) + ((uN.x - uC.x) - (uC.x - uS.x))) * inv_h2 - k2 * uC.x;
  r.y = -(((uE.y - uC.y) - (uC.y - uW.y)) + ((uN.y - uC.y) - (uC.y - uS.y))) * inv_h2 - k2 * uC.y;
  return r;
}

// Only the x factors differ from 1 (s_y(j) = 1/s_y(j +- 1/2) = 1 exactly): the general form with
// its exact products by 1 dropped.
template <typename R>
__device__ __forceinline__ C<R> stencil_point_xpml(C<R> uC, C<R> uE, C<R> uW, C<R> uN, C<R> uS, C<R> sxi, C<R> ixm,
                                                   C<R> ixp, R k2, R inv_h2) {
  C<R> fx = csub(cmul(csub(uE, uC), ixp), cmul(csub(uC, uW), ixm));
  C<R> fy = csub(csub(uN, uC), csub(uC, uS));
  C<R> acc = cadd(fx, cmul(sxi, fy));
  C<R> diag = cmul(sxi, uC);
  C<R> r;
  r.x = -acc.x * inv_h2 - k2 * diag.x;
  r.y = -acc.y * inv_h2 - k2 * diag.y;
  return r;
}

// Only the y factors differ from 1.
template <typename R>
__device__ __forceinline__ C<R> stencil_point_ypml(C<R> uC, C<R> uE, C<R> uW, C<R> uN, C<R> uS, C<R> syj, C<R> iym,
                                                   C<R> iyp, R k2, R inv_h2) {
  C<R> fx = csub(csub(uE, uC), csub(uC, uW));
  C<R> fy = csub(cmul(csub(uN, uC), iyp), cmul(csub(uC, uS), iym));
  C<R> acc = cadd(cmul(syj, fx), fy);
  C<R> diag = cmul(syj, uC);
  C<R> r;
  r.x = -acc.x * inv_h2 - k2 * diag.x;
  r.y = -acc.y * inv_h2 - k2 * diag.y;
  return r;
}

// The cheapest exact form for the point: xunit / yunit say whether all x / y factors are 1.
template <typename R>
__device__ __forceinline__ C<R> stencil_point_any(bool xunit, bool yunit, C<R> uC, C<R> uE, C<R> uW, C<R> uN, C<R> uS,
                                                  C<R> sxi, C<R> ixm, C<R> ixp, C<R> syj, C<R> iym, C<R> iyp, R k2,
                                                  R inv_h2) {
  if (xunit && yunit) return stencil_point_unit<R>(uC, uE, uW, uN, uS, k2, inv_h2);
  if (yunit) return stencil_point_xpml<R>(uC, uE, uW, uN, uS, sxi, ixm, ixp, k2, inv_h2);
  if (xunit) return stencil_point_ypml<R>(uC, uE, uW, uN, uS, syj, iym, iyp, k2, inv_h2);
  return stencil_point<R>(uC, uE, uW, uN, uS, sxi, ixm, ixp, syj, iym, iyp, k2, inv_h2);
}

}  // namespace helm
