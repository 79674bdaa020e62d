// Camera and ray geometry shared by the sampler and the crop / ray-pool
// builder: the binary64 localisation of a pixel (Sec. 4.3, the RPC camera
// model), the binary64 -> binary32 window-local ray through a pixel centre,
// and the binary32 slab clip and window acceptance (Sec. 4.4).  Every value
// that decides something discrete is a fixed sequence of IEEE operations
// with explicit round-to-nearest intrinsics (no fused multiply-add).
#pragma once
#include "common.cuh"

namespace snk {

// ---- camera (binary64) -----------------------------------------------------
__device__ __forceinline__ double rpc_poly(const double *k, double c, double r, double h) {
  // monomials 1, c, r, h, cr, ch, rh, c^2, r^2, h^2, crh, c^3, cr^2, ch^2, c^2 r,
  // r^3, rh^2, c^2 h, r^2 h, h^3; products left to right, sum left to right.
  const double cc = dmul(c, c), rr = dmul(r, r), hh = dmul(h, h);
  double s = k[0];
  s = dadd(s, dmul(k[1], c));
  s = dadd(s, dmul(k[2], r));
  s = dadd(s, dmul(k[3], h));
  s = dadd(s, dmul(k[4], dmul(c, r)));
  s = dadd(s, dmul(k[5], dmul(c, h)));
  s = dadd(s, dmul(k[6], dmul(r, h)));
  s = dadd(s, dmul(k[7], cc));
  s = dadd(s, dmul(k[8], rr));
  s = dadd(s, dmul(k[9], hh));
  s = dadd(s, dmul(k[10], dmul(dmul(c, r), h)));
  s = dadd(s, dmul(k[11], dmul(cc, c)));
  s = dadd(s, dmul(k[12], dmul(c, rr)));
  s = dadd(s, dmul(k[13], dmul(c, hh)));
  s = dadd(s, dmul(k[14], dmul(cc, r)));
  s = dadd(s, dmul(k[15], dmul(rr, r)));
  s = dadd(s, dmul(k[16], dmul(r, hh)));
  s = dadd(s, dmul(k[17], dmul(cc, h)));
  s = dadd(s, dmul(k[18], dmul(rr, h)));
  s = dadd(s, dmul(k[19], dmul(hh, h)));
  return s;
}

__device__ __forceinline__ void localise(const DevView &v, double row, double col, double h, double &x, double &y) {
  if (v.kind == SNK_CAM_AFFINE) {
    x = dadd(dadd(dadd(v.a[0], dmul(v.a[1], col)), dmul(v.a[2], row)), dmul(v.a[3], h));
    y = dadd(dadd(dadd(v.b[0], dmul(v.b[1], col)), dmul(v.b[2], row)), dmul(v.b[3], h));
    return;
  }
  const double rn = ddiv(dsub(row, v.off[0]), v.scale[0]);
  const double cn = ddiv(dsub(col, v.off[1]), v.scale[1]);
  const double hn = ddiv(dsub(h, v.off[2]), v.scale[2]);
  x = dadd(v.off[3], dmul(v.scale[3], ddiv(rpc_poly(v.coef[0], cn, rn, hn), rpc_poly(v.coef[1], cn, rn, hn))));
  y = dadd(v.off[4], dmul(v.scale[4], ddiv(rpc_poly(v.coef[2], cn, rn, hn), rpc_poly(v.coef[3], cn, rn, hn))));
}

// ---- slab clip (binary32) ----------------------------------------------------
struct Slab {
  float t_in, t_out;
};

__device__ __forceinline__ Slab slab(const float o[3], const float d[3], const float inv[3], const float lo[3],
                                     const float hi[3]) {
  float tn[3], tf[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (d[a] == 0.0f) {
      const bool inside = o[a] >= lo[a] && o[a] <= hi[a];
      tn[a] = inside ? -INFINITY : INFINITY;
      tf[a] = inside ? INFINITY : -INFINITY;
    } else {
      const float t1 = fmul(fsub(lo[a], o[a]), inv[a]);
      const float t2 = fmul(fsub(hi[a], o[a]), inv[a]);
      tn[a] = fminf(t1, t2);
      tf[a] = fmaxf(t1, t2);
    }
  }
  Slab s;
  s.t_in = fmaxf(fmaxf(fmaxf(0.0f, tn[0]), tn[1]), tn[2]);
  s.t_out = fminf(fminf(tf[0], tf[1]), tf[2]);
  return s;
}

// Window-local binary32 ray through the centre of pixel (row, col): the line through the pixel's
// localisations at z_max and z_min (binary64), origin at z_max minus the window origin, unit direction.
__device__ __forceinline__ void pixel_ray(const DevView &cv, int row, int col, const WinParams &win, float o[3],
                                          float d[3]) {
  const double rr = dadd((double)row, 0.5), cc = dadd((double)col, 0.5);
  double xt, yt, xb, yb;
  localise(cv, rr, cc, win.z_max, xt, yt);
  localise(cv, rr, cc, win.z_min, xb, yb);
  const double Dx = dsub(xb, xt), Dy = dsub(yb, yt), Dz = dsub(win.z_min, win.z_max);
  const double n = __dsqrt_rn(dadd(dadd(dmul(Dx, Dx), dmul(Dy, Dy)), dmul(Dz, Dz)));
  o[0] = __double2float_rn(dsub(xt, win.origin[0]));
  o[1] = __double2float_rn(dsub(yt, win.origin[1]));
  o[2] = __double2float_rn(dsub(win.z_max, win.origin[2]));
  d[0] = __double2float_rn(ddiv(Dx, n));
  d[1] = __double2float_rn(ddiv(Dy, n));
  d[2] = __double2float_rn(ddiv(Dz, n));
}

// Acceptance (Sec. 4.4): the ray meets the scene box and its scene interval lies inside the
// window box.  Also returns 1/d (inf for d == 0) and the scene interval.
__device__ __forceinline__ bool window_accepts(const float o[3], const float d[3], const WinParams &win, float inv[3],
                                               Slab &sc) {
#pragma unroll
  for (int a = 0; a < 3; ++a) inv[a] = d[a] == 0.0f ? INFINITY : fdiv(1.0f, d[a]);
  const float zero3[3] = {0.f, 0.f, 0.f};
  sc = slab(o, d, inv, win.scene_lo, win.scene_hi);
  const Slab wn = slab(o, d, inv, zero3, win.win_hi);
  return sc.t_in < sc.t_out && wn.t_in <= sc.t_in && sc.t_out <= wn.t_out;
}

}  // namespace snk
