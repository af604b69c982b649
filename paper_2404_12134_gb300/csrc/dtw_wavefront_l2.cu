// DTW wavefront instances: R = 16, no band, l2-norm local cost.
#include "dtw_wavefront_impl.cuh"

WTS_WF_ENTRY(l2, 16, false, kCostL2)
