// Instantiations of the fused pass and the sparse extraction for double arithmetic.
#include "pass_impl.cuh"

namespace rpca {

#define RPCA_CASE(RR) \
  case RR:            \
    return launch_pass_t<double, RR>(a, s);
cudaError_t launch_pass_f64(int R, const PassArgs& a, cudaStream_t s) {
  switch (R) { RPCA_FOR_EACH_R(RPCA_CASE) }
  return cudaErrorInvalidValue;
}
#undef RPCA_CASE

#define RPCA_CASE(RR) \
  case RR:            \
    return launch_extract_count_t<double, RR>(a, s);
cudaError_t launch_extract_count_f64(int R, const ExtractArgs& a, cudaStream_t s) {
  switch (R) { RPCA_FOR_EACH_R(RPCA_CASE) }
  return cudaErrorInvalidValue;
}
#undef RPCA_CASE

#define RPCA_CASE(RR) \
  case RR:            \
    return launch_extract_write_t<double, RR>(a, s);
cudaError_t launch_extract_write_f64(int R, const ExtractArgs& a, cudaStream_t s) {
  switch (R) { RPCA_FOR_EACH_R(RPCA_CASE) }
  return cudaErrorInvalidValue;
}
#undef RPCA_CASE

#define RPCA_CASE(RR)                                                                   \
  case RR:                                                                              \
    return PassGeom{PassCfg<double, RR>::BH, PassCfg<double, RR>::BW, PassCfg<double, RR>::TM,      \
                    PassCfg<double, RR>::VW, PassLayout<double, RR>::SMEM};
PassGeom pass_geometry_f64(int R) {
  switch (R) { RPCA_FOR_EACH_R(RPCA_CASE) }
  return PassGeom{0, 0, 0, 0, 0};
}
#undef RPCA_CASE

}  // namespace rpca
