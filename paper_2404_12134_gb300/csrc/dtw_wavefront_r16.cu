// DTW wavefront instances: R = 16, no band, squared l2 local cost.
#include "dtw_wavefront_impl.cuh"

WTS_WF_ENTRY(r16, 16, false, kCostSqEuclid)
