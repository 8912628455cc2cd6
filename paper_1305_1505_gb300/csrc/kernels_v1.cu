// Radix schedule 1 of the x and y passes (fft.cuh ShapeBase<N, 1>): the
// same passes as kernels.cu with another split of each line length, compiled
// in a translation unit of their own (the tile tuner times both schedules).
#include "passes_xy.cuh"

namespace pin {

#define PIN_SIZES_V1(X) X(8) X(16) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512) X(768)

cudaError_t upload_constant_twiddles_v1() { return upload_tw_table_here(); }

cudaError_t prepare_xy_v1(int n) {
  switch (n) {
#define CASE(N) case N: return set_attrs_xy_all<N, 1>();
    PIN_SIZES_V1(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

int xy_tile_options_v1(int n, int* opts) {
  switch (n) {
#define CASE(N)                                             \
  case N:                                                   \
    opts[0] = Tiles<N, 1>::T0;                              \
    opts[1] = Tiles<N, 1>::T1;                              \
    return Tiles<N, 1>::T1 != Tiles<N, 1>::T0 ? 2 : 1;
    PIN_SIZES_V1(CASE)
#undef CASE
    default: return 0;
  }
}

PassShape pass_shape_xy_v1(int n) {
  switch (n) {
#define CASE(N) case N: return xy_shape_of<N, 1>();
    PIN_SIZES_V1(CASE)
#undef CASE
    default: return PassShape{};
  }
}

cudaError_t launch_x_v1(int n, int tc, const ArgsX& a, cudaStream_t st) {
  switch (n) {
#define CASE(N) case N: return launch_x_v<N, 1>(tc, a, st);
    PIN_SIZES_V1(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_y_v1(int n, int tc, const ArgsY& a, cudaStream_t st) {
  switch (n) {
#define CASE(N) case N: return launch_y_v<N, 1>(tc, a, st);
    PIN_SIZES_V1(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pin
