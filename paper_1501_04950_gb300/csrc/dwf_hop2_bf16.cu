// Instantiation of the tuned hopping pass (dwf_hop2.cuh) for one storage precision;
// one translation unit per precision so the build compiles them in parallel.
#include "dwf_hop2.cuh"

DWF_HOP2_INSTANTIATE(launch_hop2_bf16, Store16<true>)
