// One (N, QC, QV) instantiation of the libdgcns kernels; compiled once per
// entry of DGCNS_CONFIGS with -DINST_N=.. -DINST_QC=.. -DINST_QV=.. so that the
// configurations build in parallel.
#include "dg_launch.cuh"

#define DGCNS_CAT3(a, b, c) launchers_##a##_##b##_##c
#define DGCNS_NAME(a, b, c) DGCNS_CAT3(a, b, c)

namespace dgcns {
Launchers DGCNS_NAME(INST_N, INST_QC, INST_QV)() { return make_launchers<INST_N, INST_QC, INST_QV>(); }
}  // namespace dgcns
