// Solid nodes (general geometry): from a byte mask of solid nodes, the
// per-cell link bits the step kernels read (Domain::solid).  Bit a of a
// fluid cell is set when the pull source x - c_a of link a -- after the
// periodic wrap and the symmetry mirror of the box faces, and not beyond a
// wall, which bounces back already -- is a solid node; a solid cell gets
// kSolidCell.  A link with a solid source bounces back as off a wall at rest
// halfway between the two nodes.
#include "lbm_internal.h"
#include "lbm_kernels.cuh"

namespace lbm {
namespace {

template <int Q>
__global__ void k_solid_links(int nx, int ny, int nz, int per, int sym,
                              const uint8_t* __restrict__ bytes, uint32_t* __restrict__ links) {
  const int64_t N = (int64_t)nx * ny * nz;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    links[i] = solid_link_bits<Q>(nx, ny, nz, per, sym, bytes, i);
}

}  // namespace

cudaError_t launch_solid_links(const DomainDesc& d, const uint8_t* bytes, uint32_t* links,
                               cudaStream_t st) {
  const int per = d.per[0] | (d.per[1] << 1) | (d.per[2] << 2);
  const int64_t blocks64 = (d.N + 255) / 256;
  const int blocks = (int)(blocks64 < 8192 ? blocks64 : 8192);
  if (d.Q == 14) k_solid_links<14><<<blocks, 256, 0, st>>>(d.nx, d.ny, d.nz, per, d.sym, bytes, links);
  else if (d.Q == 18) k_solid_links<18><<<blocks, 256, 0, st>>>(d.nx, d.ny, d.nz, per, d.sym, bytes, links);
  else k_solid_links<26><<<blocks, 256, 0, st>>>(d.nx, d.ny, d.nz, per, d.sym, bytes, links);
  return cudaGetLastError();
}

}  // namespace lbm
