// Host-side internals shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/lbm.h"

namespace lbm {

// Number of FP64 statistics a reduction produces (layout of lbm_stats after
// the two step counters): 3 du, 3 u, 3 u_prev, P, 3 flux, max, nonfinite.
constexpr int kNumSums = 14;   // summed entries
constexpr int kNumStats = 15;  // plus the max
constexpr int kReduceBlocks = 1216;  // 8 x 152 SMs; partials per reduction
constexpr int kReduceThreads = 256;

// Everything a kernel needs to know about one domain, in FP64; the launchers
// convert it to the arithmetic type of the storage.
struct DomainDesc {
  int Q, nx, ny, nz, storage;
  int64_t N;
  void* f;
  int per[3];
  int moving;  // bit f: face f is a moving wall
  int sym;     // bit f: face f is a symmetry plane
  int neq_vel; // bit f: face f is a non-equilibrium extrapolation velocity face
  int neq_pre; // bit f: ... pressure face
  double p_face[6], p_amp[6], p_period;  // pressure of the pressure faces
  const uint32_t* solid;  // device: per-cell solid-link bits (Domain::solid), or null
  double uw[6][3];
  int edge_axis[6];  // edge profiles of moving faces (lbm_geom)
  double edge_scale[6][2];
  double s[6];  // sc, se, sq, snu, spi, st
  double force[3];
  double period;
  double p_ref;
  int rounding;  // enum lbm_rounding
};

struct BlockShape {
  int bx, by;
  int cpt;      // cells per thread: 1, or 2 (pairs along x, FP32 arithmetic only)
  int pdl = 1;  // programmatic dependent launch of consecutive steps
};

BlockShape default_block(int nx, int ny);

// The face fields of d (per, moving, sym, neq_*, uw) from a geometry.
// Returns nullptr, or the reason the geometry is invalid (then d is
// unchanged).  d's sizes must be set (extrapolation faces need 3 nodes).
const char* set_faces(DomainDesc& d, const lbm_geom* g);

// Per-cell solid-link bits (Domain::solid) of the solid-node mask `bytes`
// (N device bytes, nonzero = solid) for d's geometry.
cudaError_t launch_solid_links(const DomainDesc& d, const uint8_t* bytes, uint32_t* links,
                               cudaStream_t st);

// Non-equilibrium extrapolation of the boundary nodes of d's LBM_NEQ_*
// faces, on the populations of step n (after the step n-1 -> n).
cudaError_t launch_neq(const DomainDesc& d, int64_t n, cudaStream_t st);

// Message returned by lbm_last_error() on the calling thread.
void set_last_error(const std::string& msg);

// F(t_n) of a domain.
void force_at(const DomainDesc& d, int64_t n, double F[3]);

// Queue one fused step n -> n+1 (parity n & 1).
cudaError_t launch_step(const DomainDesc& d, int64_t n, BlockShape b, cudaStream_t st);

// f = f_eq(p - p_ref, u) at every node, stored for step 0 (even layout).
cudaError_t launch_init(const DomainDesc& d, const double* u, const double* p,
                        cudaStream_t st);

// Canonical populations / u / p of step n into a device buffer.
cudaError_t launch_read(const DomainDesc& d, int64_t n, unsigned mask, void* dst,
                        int dtype, cudaStream_t st);

// Canonical FP64 populations into the storage layout of step n.
cudaError_t launch_write(const DomainDesc& d, int64_t n, const double* src,
                         cudaStream_t st);

// FP64 reductions at step n against the snapshot u_prev (valid if
// have_prev); writes the new snapshot if u_prev != nullptr, per-block
// partials to `partials` (kReduceBlocks * kNumStats doubles) and the final
// statistics (kNumStats doubles) to `out`.
cudaError_t launch_reduce(const DomainDesc& d, int64_t n, double* u_prev,
                          int have_prev, double* partials, double* out,
                          cudaStream_t st);

}  // namespace lbm
