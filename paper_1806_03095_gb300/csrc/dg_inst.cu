// One part of one (N, QC, QV) instantiation of the libdgcns kernels; compiled once per entry of
// DGCNS_CONFIGS and part 0..DGCNS_PARTS-1 with -DINST_N=.. -DINST_QC=.. -DINST_QV=.. -DINST_PART=..
// so that everything builds in parallel.
#include "dg_launch.cuh"

#define DGCNS_CAT4(a, b, c, d) launchers_##a##_##b##_##c##_##d
#define DGCNS_NAME(a, b, c, d) DGCNS_CAT4(a, b, c, d)

namespace dgcns {
void DGCNS_NAME(INST_N, INST_QC, INST_QV, INST_PART)(Launchers& L) {
  fill_launchers<INST_N, INST_QC, INST_QV, INST_PART>(L);
}
}  // namespace dgcns
