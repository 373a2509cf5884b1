// Instantiations of the fused pass and the sparse extraction for float arithmetic.
#include "pass_impl.cuh"

namespace rpca {

#define RPCA_CASE(RR) \
  case RR:            \
    return launch_pass_t<float, RR>(a, s);
cudaError_t launch_pass_f32(int R, const PassArgs& a, cudaStream_t s) {
  switch (R) { RPCA_FOR_EACH_R(RPCA_CASE) }
  return cudaErrorInvalidValue;
}
#undef RPCA_CASE

#define RPCA_CASE(RR) \
  case RR:            \
    return launch_extract_count_t<float, RR>(a, s);
cudaError_t launch_extract_count_f32(int R, const ExtractArgs& a, cudaStream_t s) {
  switch (R) { RPCA_FOR_EACH_R(RPCA_CASE) }
  return cudaErrorInvalidValue;
}
#undef RPCA_CASE

#define RPCA_CASE(RR) \
  case RR:            \
    return launch_extract_write_t<float, RR>(a, s);
cudaError_t launch_extract_write_f32(int R, const ExtractArgs& a, cudaStream_t s) {
  switch (R) { RPCA_FOR_EACH_R(RPCA_CASE) }
  return cudaErrorInvalidValue;
}
#undef RPCA_CASE

#define RPCA_CASE(RR) \
  case RR:            \
    return launch_extract_words_t<RR>(a, words, cc, nw, s);
cudaError_t launch_extract_words_f32(int R, const ExtractArgs& a, const unsigned* words, const unsigned* cc, int nw,
                                     cudaStream_t s) {
  switch (R) { RPCA_FOR_EACH_R(RPCA_CASE) }
  return cudaErrorInvalidValue;
}
#undef RPCA_CASE

#define RPCA_CASE(RR)                                                                   \
  case RR:                                                                              \
    return PassGeom{PassCfg<float, RR>::BH, PassCfg<float, RR>::BW, PassCfg<float, RR>::TM,      \
                    PassCfg<float, RR>::VW, PassLayout<float, RR>::SMEM};
PassGeom pass_geometry_f32(int R) {
  switch (R) { RPCA_FOR_EACH_R(RPCA_CASE) }
  return PassGeom{0, 0, 0, 0, 0};
}
#undef RPCA_CASE

}  // namespace rpca
