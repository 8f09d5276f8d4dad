// sg_kernels.cuh -- all CUDA kernels of the sparse-grid WENO5 hot path, templated on the state
// precision T (double or float) and the dimension.
//
// Instantiated twice:
//   sg_kernels_f64.cu, compiled with --fmad=false: every double expression is then a fixed
//     sequence of IEEE-754 operations in the order the paper prints the formula, so the FP64
//     path reproduces a plain sequential evaluation bit for bit;
//   sg_kernels_f32.cu, with contraction on: the float path uses an algebraically equivalent
//     reformulation with fewer operations and a compensated state.
#pragma once
#include "sg_weno.cuh"
#include "sg_stage.cuh"
#include "sg_stage_line.cuh"
#include "sg_sweep2.cuh"
#include "sg_aux.cuh"
#include "sg_combine2.cuh"
