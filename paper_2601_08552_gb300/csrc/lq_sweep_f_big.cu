// lq_sweep_f_big.cu -- the sweep kernel instance for FP32 panels (both mixed modes), more than 32 particles per spin.
#include "lq_sweep.cuh"

LQ_SWEEP_INSTANCE(float, true, f_big)
