// Persistent ring-buffer H psi kernel for FP32 blocks of 32 states (see
// stencil_ring.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "common.h"

namespace rs {

struct RingPlan;

// Builds the kernel's tables from the host grid, the point-major nonlocal
// tables (coff [npts+1], catom / cg32 [entries] with four projector values
// per entry), the FP32 potential, the FP32 centre weight of the star, the
// number of atoms and the z-slab height
// of a work unit.  Returns RS_OK with *out == nullptr when the grid cannot
// use the kernel (2^28 points or more, a plane record or a CTA's unit list
// above the shared-memory budget).
int ring_plan_build(RingPlan **out, const rs_grid *g, const std::vector<int32_t> &coff, const std::vector<int32_t> &catom,
                    const std::vector<float> &cg32, const std::vector<float> &v32, float w0, int n_atoms, int slab);
void ring_plan_destroy(RingPlan *p);

// True when the kernel takes this block: nb a multiple of 32 and 16-byte
// copies of psi rows (16-byte aligned base, ld a multiple of 4).
bool ring_usable(const RingPlan *p, const float *psi, int64_t ldp, int nb);

// Hpsi = (T + V + V_nl) psi for nb states (w: kinetic weights, cproj: the
// projection coefficients [atom][nb][4] of this block, already computed).
int ring_launch(RingPlan *p, const float *psi, int64_t ldp, float *hpsi, int64_t ldh, const float *cproj, int nb,
                const float w[5], cudaStream_t st);

// Status word of the kernel's bounded waits (0 = none timed out); blocking.
int ring_status(const RingPlan *p, int *flag);
// Rewrites the plan's potential values from a new FP32 potential [npts]
// (asynchronous).
int ring_set_potential(RingPlan *p, const float *v32, cudaStream_t st);
// Clears the status word (blocking).
int ring_reset_status(RingPlan *p);
// Device address of the status word (nullptr without a plan).
int *ring_status_word(RingPlan *p);
// Barrier tests before a wait gives up (tests < 0: the default).
void ring_set_wait_limit(RingPlan *p, int tests);

}  // namespace rs
