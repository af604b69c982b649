// DTW wavefront instances: R = 16, Sakoe-Chiba band, l2-norm local cost.
#include "dtw_wavefront_impl.cuh"

WTS_WF_ENTRY(l2b, 16, true, kCostL2)
