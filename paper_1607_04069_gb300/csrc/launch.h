// launch.h -- host-side launchers of the device kernels (internal to the library).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace pg {

constexpr int kMoverThreads = 256;
#ifndef PG_MOVER_MIN_BLOCKS
#define PG_MOVER_MIN_BLOCKS 2
#endif
constexpr int kMoverMinBlocks = PG_MOVER_MIN_BLOCKS;   // resident CTAs per SM the register budget is sized for
#ifndef PG_MOVER_PDL
#define PG_MOVER_PDL 1
#endif
constexpr int kMoverPdl = PG_MOVER_PDL;           // step launches overlap the previous launch's tail
constexpr int kTpThreads = 256;
#ifndef PG_TP_MIN_BLOCKS
#define PG_TP_MIN_BLOCKS 3
#endif
constexpr int kTpMinBlocks = PG_TP_MIN_BLOCKS;   // resident CTAs per SM the TP step's registers are sized for

size_t mover_smem(int ncell);
size_t tp_smem(int ncell);
cudaError_t mover_occupancy(const Dev& d, int* blocks_per_sm);
// initial loading of n particles with ids tag | (id0 + k)
cudaError_t launch_init(const Dev& d, int s, long long n, long long id0, float vth, cudaStream_t st);
// mode 0: one PIC/MCC step; mode 1: deposit the current state and solve the field
cudaError_t launch_mover(const Dev& d, const StepArgs& a, int grid, int mode, cudaStream_t st);
// one step of every discharge of a batch (32-bit positions); sample: the launch
// samples the flux moments and the EEDF of every member.  mover_batch_attr
// must have been called with max_ncell first.
cudaError_t launch_mover_batch(const BatchEntry* ent, const int* owner, int grid, int max_ncell, bool sample,
                               cudaStream_t st);
// the same with resident CTAs taking chunks of CTA slots from the work counter
// work[2] (zero before the first launch; each launch leaves it zero)
cudaError_t launch_mover_batch_chunks(const BatchEntry* ent, const BatchChunk* chunks, int nchunks, unsigned int* work,
                                      int grid, int max_ncell, bool sample, cudaStream_t st);
// the shared-memory attribute of both batch instantiations (set before a graph
// capture), and the resident CTAs per SM it allows (blocks_per_sm may be NULL)
cudaError_t mover_batch_attr(int max_ncell, int* blocks_per_sm);
// FP64 field/potential of the current state; accumulate != 0 also adds the
// current step to the time averages if no step launch has done so yet
cudaError_t launch_field(const Dev& d, double v_left, int accumulate, cudaStream_t st);
// first null-collision candidate step of n uploaded particles that are first pushed at step l0
cudaError_t launch_entry_nev(const Dev& d, int s, unsigned int half, long long n, unsigned int l0, cudaStream_t st);
cudaError_t launch_sort(const Dev& d, int s, int grid, cudaStream_t st);
// one TP step; sample: the step adds to the time averages (thinned-candidate
// mode: only then does the launch carry the tallies in shared memory)
cudaError_t launch_tp_step(const Dev& d, int grid, bool sample, cudaStream_t st);
// resident CTAs per SM of the TP step kernel of d's collision mode and law,
// for a sample step or another
cudaError_t tp_occupancy(const Dev& d, bool sample, int* blocks_per_sm);
// event-driven flight: every live TP atom through at most kmax events; the
// atoms still alive are added to Ctl::tpf_alive
cudaError_t launch_tp_flight(const Dev& d, int kmax, long long n, cudaStream_t st);
cudaError_t launch_tp_launch(const Dev& d, long long n, long long id0, float Emax, cudaStream_t st);
cudaError_t launch_op_deposit(const void* pos, int pos64, long long n, int ncell, int kshift,
                              unsigned long long* q, int grid, cudaStream_t st);
// record the detail that pic_last_error reports on the calling thread
void set_last_error(const char* msg);
cudaError_t launch_op_poisson(const long long* qi, const long long* qe, int N, double A, double inv_dx,
                              double v_left, double* phi, double* E64, cudaStream_t st);

}  // namespace pg
