// Hard-min band wavefront for DTW (Eq. 1 via Eq. 5 with gamma = 0): the
// dispatch between the instance sets.  The kernels and the algorithm are in
// dtw_wavefront_impl.cuh; each set is compiled by its own dtw_wavefront_*.cu.
#include "dtw_wavefront.cuh"

namespace wts {

cudaError_t launch_dtw_wavefront(int mode, int D, int R, const DPParams& p, int grid, int block, cudaStream_t st)
{
    if (p.cost_kind == kCostL2) {
        if (R != 16) return cudaErrorInvalidValue;
        return p.banded ? wf_launch_l2b(mode, D, p, grid, block, st) : wf_launch_l2(mode, D, p, grid, block, st);
    }
    if (p.cost_kind != kCostSqEuclid) return cudaErrorInvalidValue;
    if (p.banded) return R == 16 ? wf_launch_r16b(mode, D, p, grid, block, st) : cudaErrorInvalidValue;
    switch (R) {
        case 4: return wf_launch_r4(mode, D, p, grid, block, st);
        case 8: return wf_launch_r8(mode, D, p, grid, block, st);
        case 16: return wf_launch_r16(mode, D, p, grid, block, st);
        case 32: return wf_launch_r32(mode, D, p, grid, block, st);
        default: return cudaErrorInvalidValue;
    }
}

int dtw_wavefront_max_blocks_per_sm(int mode, int D, int R, int block, int banded, int cost_kind)
{
    if (cost_kind == kCostL2) {
        if (R != 16) return 0;
        return banded ? wf_occ_l2b(mode, D, block) : wf_occ_l2(mode, D, block);
    }
    if (cost_kind != kCostSqEuclid) return 0;
    if (banded) return R == 16 ? wf_occ_r16b(mode, D, block) : 0;
    switch (R) {
        case 4: return wf_occ_r4(mode, D, block);
        case 8: return wf_occ_r8(mode, D, block);
        case 16: return wf_occ_r16(mode, D, block);
        case 32: return wf_occ_r32(mode, D, block);
        default: return 0;
    }
}

}  // namespace wts
