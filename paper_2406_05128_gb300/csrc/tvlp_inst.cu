// One explicit instantiation of the kernels and launchers, selected by
// -DTVLP_SCALAR=<float|double> -DTVLP_MP=<padded order> at compile time.
#include "tvlp_impl.cuh"

#ifndef TVLP_SCALAR
#error "define TVLP_SCALAR"
#endif
#ifndef TVLP_MP
#error "define TVLP_MP"
#endif

template struct tvlp::Impl<TVLP_SCALAR, TVLP_MP>;
