// persist.cuh -- one persistent launch per direction for a batch of uneven problems.
//
// The batched classes of a batch (FP32, grids up to 2^18 points) are normally run with
// two launches per class and direction.  The persistent kernel runs all of them in one
// launch: a grid of about as many 256-thread CTAs as fit on the GPU pulls work items
// from one queue by an atomic ticket.  An item is the work one CTA of a class launch
// would do -- (problem, block) of the first pass (pass 1, or pass A), or of the second
// (pass 2, or pass B).  Every first-pass item of every problem comes before any
// second-pass item in the queue, and a second-pass item first waits until its problem's
// first-pass items are all done (a per-problem counter).  Each counted item was taken
// from the queue by a running CTA before the waiting one took its own, so the wait
// always ends; it is still bounded by time (2 s of %globaltimer), after which the
// problem's error word records a timeout (nufft_batch_check reports it) and the CTA
// goes on.  The last CTA to leave resets the ticket and the counters for the next launch.
//
// A CTA has 256 threads whatever the class: the row passes run with 256 / TT teams
// (idle teams only meet the barriers), and the column passes of small grids, which need
// fewer threads, let the extra threads shadow a role (pass 1 and pass B write the same
// values to the same places from both).  Items use the class arguments built at plan time
// (each member's own plan: its buffers, K, tables); the coefficient tables are stored
// 16 x 16 (zero-padded) and staged per item at the class's rank bound, for which the row
// passes are compiled (8, 12, 16).
#pragma once

#include "passes.cuh"

namespace nufft {

struct PItem {
    int kind;    // 0: first pass (pass 1 / pass A), 1: second pass (pass 2 / pass B)
    int cls;     // index into the class table
    int member;  // the problem's index within its class (its argument entry)
    int prob;    // the problem's index in the batch (its counter and coefficients)
    int bx, by;  // the first block the class launch would have given a CTA
    int nbx;     // consecutive blocks bx .. bx + nbx - 1 (same by) that this item runs
};

struct PClass {
    int P_rows, P_cols;                      // row FFT length (L1), column FFT length (L2)
    int km;                                  // the row passes' rank bound: 8, 12 or 16
    const PassArgs<float> *args[2];          // per member: first pass, second pass
};

// The device state of one direction of a persistent batch.
struct PState {
    const PItem *items;
    int n_items;
    const PClass *classes;
    const Beta<float, 16> *betas;   // per problem, 16 x 16 zero-padded
    int *done;                      // per problem: first-pass items finished
    const int *need;                // per problem: its first-pass item count
    int *ctl;                       // [0] ticket, [1] CTAs that have left
    int nprob;
};

// Launch one direction (0: forward, 1: adjoint) of a persistent batch: grid CTAs of 256
// threads, smem bytes of dynamic shared memory (persist_fwd.cu, persist_adj.cu).
int launch_persistent_fwd(const PState &st, int grid, size_t smem, const ManyIO &io, cudaStream_t s);
int persistent_blocks_fwd(size_t smem, int *out);
int launch_persistent(int dir, const PState &st, int grid, size_t smem, const ManyIO &io, cudaStream_t s);
// The CTAs of one direction's kernel that fit on the device at once (per SM), for smem.
int persistent_blocks_per_sm(int dir, size_t smem, int *out);

}  // namespace nufft
