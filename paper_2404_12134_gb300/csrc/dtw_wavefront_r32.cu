// DTW wavefront instances: R = 32 (d <= 3), no band, squared l2 local cost.
#include "dtw_wavefront_impl.cuh"

WTS_WF_ENTRY(r32, 32, false, kCostSqEuclid)
