// Observables read from the density: the dipole in the length gauge of a
// periodic box (the sawtooth coordinate r_a - L/2, r_a = i h in [0, L), of
// the field workload along each axis), for the vibrational and infrared
// analysis of trajectories.

#include "emd_internal.cuh"

namespace {

// part[a * nblocks + b] = block b's sum of rho(r) (r_a - L/2), a = x, y, z
__global__ void __launch_bounds__(256)
k_dipole(int n, double h, const double *__restrict__ rho, double *__restrict__ part) {
  __shared__ double red[8 * 3];
  const int n3 = n * n * n;
  const double half = 0.5 * n * h;
  double acc[3] = {0.0, 0.0, 0.0};
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n3; p += gridDim.x * blockDim.x) {
    const int x = p % n, y = (p / n) % n, z = p / (n * n);
    const double r = rho[p];
    acc[0] += r * (x * h - half);
    acc[1] += r * (y * h - half);
    acc[2] += r * (z * h - half);
  }
  emd_block_sum<3>(acc, red);
  if (threadIdx.x == 0)
    for (int a = 0; a < 3; ++a) part[a * gridDim.x + blockIdx.x] = acc[a];
}

}  // namespace

void emd_launch_dipole_partials(int n, double h, const double *rho, double *part, int nblocks,
                                cudaStream_t st) {
  emd_note_launches(1);
  k_dipole<<<nblocks, 256, 0, st>>>(n, h, rho, part);
}
