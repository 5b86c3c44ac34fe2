// The persistent solve kernel in the 512-thread block shape (16 warps, one
// CTA per SM), as tac::wide::solve_kernel: every phase of a pad's solve
// spreads over twice the threads of the 256-thread shape. It serves batches
// with fewer pads than the GPU has CTA slots, where one 256-thread CTA per
// pad leaves most of each SM idle; tac_set_block_shape and
// tac_autotune_block_shape choose between the shapes.
#define TAC_WIDE 1
#include "kernels.cu"
