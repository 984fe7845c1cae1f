// lq_sweep_f_small.cu -- the sweep kernel instance for FP32 panels (both mixed modes), up to 32 particles per spin.
#include "lq_sweep.cuh"

LQ_SWEEP_INSTANCE(float, false, f_small)
