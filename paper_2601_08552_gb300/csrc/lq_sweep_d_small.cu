// lq_sweep_d_small.cu -- the sweep kernel instance for FP64 panels, up to 32 particles per spin.
#include "lq_sweep.cuh"

LQ_SWEEP_INSTANCE(double, false, d_small)
