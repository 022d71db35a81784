// Mean kinetic energy and mean enstrophy of Sec. IV C (compressible Taylor-Green vortex):
//   KE = <rho u.u / 2>,  eps = <rho w.w / 2>,  w = curl u,
// averaged over all sites of both sublattices.  The curl is taken on each sublattice's own
// grid (unit spacing) by second-order central differences; y and z wrap, x wraps when the x
// faces are periodic and otherwise takes second-order one-sided differences at its two end
// planes.  Input: the FP64 fields of lbm_moments (rho[site], u[a * us + site], sites ordered
// sub, z, y, x).  Per-block partial sums in a fixed tree order, then one block adds them in a
// fixed order, so the result is deterministic.
#include "lbm_internal.h"

namespace lbm {
namespace {

constexpr int kDiagBlock = 256;

struct FieldView {
  int nx, ny, nz;
  int x_periodic;
  const double* u;
  long long us;
  __device__ __forceinline__ double at(int c, long long base, int x, int y, int z) const {
    return u[c * us + base + (static_cast<long long>(z) * ny + y) * nx + x];
  }
};

// d/dx of component c at (x, y, z) of the sublattice whose first site is `base`.
__device__ __forceinline__ double ddx(const FieldView& v, int c, long long base, int x, int y, int z) {
  if (v.x_periodic) {
    const int xp = x + 1 == v.nx ? 0 : x + 1, xm = x == 0 ? v.nx - 1 : x - 1;
    return 0.5 * (v.at(c, base, xp, y, z) - v.at(c, base, xm, y, z));
  }
  if (x == 0) return -1.5 * v.at(c, base, 0, y, z) + 2.0 * v.at(c, base, 1, y, z) - 0.5 * v.at(c, base, 2, y, z);
  if (x == v.nx - 1)
    return 1.5 * v.at(c, base, x, y, z) - 2.0 * v.at(c, base, x - 1, y, z) + 0.5 * v.at(c, base, x - 2, y, z);
  return 0.5 * (v.at(c, base, x + 1, y, z) - v.at(c, base, x - 1, y, z));
}
__device__ __forceinline__ double ddy(const FieldView& v, int c, long long base, int x, int y, int z) {
  const int yp = y + 1 == v.ny ? 0 : y + 1, ym = y == 0 ? v.ny - 1 : y - 1;
  return 0.5 * (v.at(c, base, x, yp, z) - v.at(c, base, x, ym, z));
}
__device__ __forceinline__ double ddz(const FieldView& v, int c, long long base, int x, int y, int z) {
  const int zp = z + 1 == v.nz ? 0 : z + 1, zm = z == 0 ? v.nz - 1 : z - 1;
  return 0.5 * (v.at(c, base, x, y, zp) - v.at(c, base, x, y, zm));
}

__global__ void __launch_bounds__(kDiagBlock) diag_partials_kernel(FieldView v, const double* rho, double* partials) {
  __shared__ double ske[kDiagBlock], sen[kDiagBlock];
  const long long n = static_cast<long long>(v.nx) * v.ny * v.nz;
  const long long k = static_cast<long long>(blockIdx.x) * kDiagBlock + threadIdx.x;
  double ke = 0.0, en = 0.0;
  if (k < 2 * n) {
    const long long base = k >= n ? n : 0;
    const long long t = k - base;
    const int x = static_cast<int>(t % v.nx);
    const int y = static_cast<int>((t / v.nx) % v.ny);
    const int z = static_cast<int>(t / (static_cast<long long>(v.nx) * v.ny));
    const double r = rho[k];
    const double ux = v.u[k], uy = v.u[v.us + k], uz = v.u[2 * v.us + k];
    const double wx = ddy(v, 2, base, x, y, z) - ddz(v, 1, base, x, y, z);
    const double wy = ddz(v, 0, base, x, y, z) - ddx(v, 2, base, x, y, z);
    const double wz = ddx(v, 1, base, x, y, z) - ddy(v, 0, base, x, y, z);
    ke = 0.5 * r * (ux * ux + uy * uy + uz * uz);
    en = 0.5 * r * (wx * wx + wy * wy + wz * wz);
  }
  ske[threadIdx.x] = ke;
  sen[threadIdx.x] = en;
  __syncthreads();
  for (int h = kDiagBlock / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      ske[threadIdx.x] += ske[threadIdx.x + h];
      sen[threadIdx.x] += sen[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = ske[0];
    partials[2 * blockIdx.x + 1] = sen[0];
  }
}

__global__ void __launch_bounds__(kDiagBlock) diag_final_kernel(const double* partials, long long nb, double inv_sites,
                                                                double* out2) {
  __shared__ double ske[kDiagBlock], sen[kDiagBlock];
  double ke = 0.0, en = 0.0;
  for (long long b = threadIdx.x; b < nb; b += kDiagBlock) {
    ke += partials[2 * b];
    en += partials[2 * b + 1];
  }
  ske[threadIdx.x] = ke;
  sen[threadIdx.x] = en;
  __syncthreads();
  for (int h = kDiagBlock / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      ske[threadIdx.x] += ske[threadIdx.x + h];
      sen[threadIdx.x] += sen[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out2[0] = ske[0] * inv_sites;
    out2[1] = sen[0] * inv_sites;
  }
}

}  // namespace

long long diagnostics_blocks(long long sites) { return (sites + kDiagBlock - 1) / kDiagBlock; }

cudaError_t launch_diagnostics(const Geometry& g, const double* rho, const double* u, long long sites,
                               double* partials, double* out2, cudaStream_t s) {
  FieldView v{g.nx, g.ny, g.nz, g.x_periodic ? 1 : 0, u, sites};
  const long long nb = diagnostics_blocks(sites);
  diag_partials_kernel<<<static_cast<unsigned int>(nb), kDiagBlock, 0, s>>>(v, rho, partials);
  diag_final_kernel<<<1, kDiagBlock, 0, s>>>(partials, nb, 1.0 / static_cast<double>(sites), out2);
  return cudaGetLastError();
}

}  // namespace lbm
