// DTW wavefront instances: rows per lane R = 8, no band, squared l2 local cost.
#include "dtw_wavefront_impl.cuh"

WTS_WF_ENTRY(r8, 8, false, kCostSqEuclid)
