// Double-float kernel terms of one source for one target, shared by the all-pairs and the
// near-field kernels. Sources are staged as float4 records (FP32 value and low part of every
// quantity, positions relative to the source drop's centre):
//   Laplace (KIND 0 target-normal double layer, 1 single layer):
//     a = (x, y, z, x_lo), b = (y_lo, z_lo, s, s_lo)
//   Stokes (KIND 2, Stokeslet on f and stresslet on u with the source normal n; KIND 3 the Stokeslet
//   alone, KIND 4 the stresslet alone):
//     a = (x, y, z, x_lo), b = (y_lo, z_lo, fx, fx_lo), c = (fy, fy_lo, fz, fz_lo),
//     d = (ux, ux_lo, uy, uy_lo), e = (uz, uz_lo, nx, nx_lo), g = (ny, ny_lo, nz, nz_lo)
// T is the target's offset from the drop centre, N0 its normal; the accumulators collect the
// kernel sums without the 1/(4 pi). Host-compilable (the CPU tests define float4 before including
// this header and compile without FMA contraction).
#pragma once

#include "dfloat.cuh"

namespace shbim {

template <int KIND>
DF_FN void df_term(const dfl::df T[3], const dfl::df N0[3], float4 a, float4 b, float4 c,
                                        float4 d, float4 e, float4 g, dfl::acc* A) {
  using dfl::df;
  const df dx = dfl::diff(T[0], df{a.x, a.w});
  const df dy = dfl::diff(T[1], df{a.y, b.x});
  const df dz = dfl::diff(T[2], df{a.z, b.y});
  const df r2 = dfl::dot3(dx, dy, dz, dx, dy, dz);
  const df ri = dfl::rsqrt(r2);
  if (KIND == 1) {
    A[0].add_prod(df{b.z, b.w}, ri);
  } else if (KIND == 0) {
    const df dn = dfl::dot3(dx, dy, dz, N0[0], N0[1], N0[2]);
    const df ri3 = dfl::mul(dfl::sqr(ri), ri);
    A[0].add_prod(dfl::mul(df{b.z, b.w}, ri3), dn);
  } else if (KIND == 4) {
    // stresslet on u alone
    const df ux{d.x, d.y}, uy{d.z, d.w}, uz{e.x, e.y};
    const df nx{e.z, e.w}, ny{g.x, g.y}, nz{g.z, g.w};
    const df hu = dfl::dot3(dx, dy, dz, ux, uy, uz);
    const df hn = dfl::dot3(dx, dy, dz, nx, ny, nz);
    const df ri2 = dfl::sqr(ri);
    const df tt = dfl::mul(dfl::mul(hu, hn), dfl::mul(dfl::mul(ri2, ri2), ri));
    A[0].add_prod(dx, tt);
    A[1].add_prod(dy, tt);
    A[2].add_prod(dz, tt);
  } else {
    // KIND 2: Stokeslet on f and stresslet on u; KIND 3: Stokeslet alone
    const df fx{b.z, b.w}, fy{c.x, c.y}, fz{c.z, c.w};
    const df hf = dfl::dot3(dx, dy, dz, fx, fy, fz);
    const df ri2 = dfl::sqr(ri);
    const df ri3 = dfl::mul(ri2, ri);
    df tt;
    if (KIND == 3) {
      tt = dfl::mul(ri3, hf);
    } else {
      const df ux{d.x, d.y}, uy{d.z, d.w}, uz{e.x, e.y};
      const df nx{e.z, e.w}, ny{g.x, g.y}, nz{g.z, g.w};
      const df hu = dfl::dot3(dx, dy, dz, ux, uy, uz);
      const df hn = dfl::dot3(dx, dy, dz, nx, ny, nz);
      tt = dfl::mul(ri3, dfl::add(hf, dfl::mul(dfl::mul(hu, hn), ri2)));
    }
    A[0].add_prod(fx, ri);
    A[0].add_prod(dx, tt);
    A[1].add_prod(fy, ri);
    A[1].add_prod(dy, tt);
    A[2].add_prod(fz, ri);
    A[2].add_prod(dz, tt);
  }
}

}  // namespace shbim
