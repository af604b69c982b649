// DTW wavefront instances: R = 16, Sakoe-Chiba band, squared l2 local cost.
#include "dtw_wavefront_impl.cuh"

WTS_WF_ENTRY(r16b, 16, true, kCostSqEuclid)
