// The assembly-free operator: the assembly operator of §3.2 Eq. 1 read degree
// of freedom by degree of freedom. Each output node gathers from its <= 8
// elements and 27 neighbours; no atomics and no assembled matrix. Mhat/Khat are
// the Q1 element matrices indexed by the XOR of the two local corner numbers.
#pragma once

#include "heat_dev.cuh"

namespace heat {

// ------------------------------------------------------------ the operator

// y at node (i,j,k) of sum_e (sa*rho_c_e*Mhat + sb*k_e*Khat) x_e, with x
// supplied by a loader ld(ii,jj,kk) for the 27 neighbours (0 outside the mesh).
template <class T, class Load>
__device__ __forceinline__ T gather_apply(const SimDev& s, T sa, T sb, int i, int j, int k, Load&& ld) {
  T v[27];
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int ii = i + dx, jj = j + dy, kk = k + dz;
        v[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)] = inside_nodes(s, ii, jj, kk) ? ld(ii, jj, kk) : T(0);
      }
  const auto* coef = coef_ptr<T>(s);
  T acc = T(0);
#pragma unroll
  for (int c = 0; c < 8; ++c) {  // node (i,j,k) is local corner c of element e
    const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
    const int ex = i - cx, ey = j - cy, ez = k - cz;
    if (ex < 0 || ey < 0 || ez < 0 || ex >= s.nx || ey >= s.ny || ez >= s.nz) continue;
    const auto cf = coef[ex + (long long)s.nx * (ey + (long long)s.ny * ez)];
    const T wa = sa * cf.x, wb = sb * cf.y;
#pragma unroll
    for (int p = 0; p < 8; ++p) {
      const int b = c ^ p;
      const int ox = (b & 1) - cx, oy = ((b >> 1) & 1) - cy, oz = ((b >> 2) & 1) - cz;
      acc += (wa * mhat<T>(s, p) + wb * khat<T>(s, p)) * v[(oz + 1) * 9 + (oy + 1) * 3 + (ox + 1)];
    }
  }
  return acc;
}


__device__ __forceinline__ void node_of(const SimDev& s, long long n, int& i, int& j, int& k) {
  const long long px = s.nx + 1, pxy = px * (s.ny + 1);
  k = (int)(n / pxy);
  const long long rem = n - (long long)k * pxy;
  j = (int)(rem / px);
  i = (int)(rem - (long long)j * px);
}

}  // namespace heat
