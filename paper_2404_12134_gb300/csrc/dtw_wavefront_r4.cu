// DTW wavefront instances: rows per lane R = 4, Sub-DTW only, squared l2 local cost.
#include "dtw_wavefront_impl.cuh"

WTS_WF_ENTRY(r4, 4, false, kCostSqEuclid)
