// lq_sweep_d_big.cu -- the sweep kernel instance for FP64 panels, more than 32 particles per spin.
#include "lq_sweep.cuh"

LQ_SWEEP_INSTANCE(double, true, d_big)
