// Mixed-precision launcher (FP32 chain + colour sum).  Placeholder: scalar FP32
// colour contraction for every basis size.
#pragma once
#include "me_kernel.cuh"
#include "me_kernel_tab.cuh"

namespace me {

template <class P> cudaError_t launch_mixed(const LaunchArgs& a)
{
    if constexpr (P::IS_TAB) return launch_tab<P, float>(a);
    else return launch_scalar<P, float>(a);
}

}  // namespace me
