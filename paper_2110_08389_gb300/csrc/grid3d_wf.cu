// grid3d_wf.cu -- the wireframe instances of the 3D warp-path kernels
// (seq3.cuh): sequences with up to WJ3_MAX ring junctions and the cuboid edge
// skeletons of Sec. 7, compiled apart from the tweed instances.
#include "seq3.cuh"

namespace tmg {

template <typename T>
cudaError_t launch_seq3_multi(const Grid3 &G, const Level3 &L, const WarpList3 &w, T *u, const T *f, cudaStream_t s) {
  return launch_warp3_t<T, true>(G, L, w, u, f, s);
}
template cudaError_t launch_seq3_multi<float>(const Grid3 &, const Level3 &, const WarpList3 &, float *, const float *,
                                              cudaStream_t);
template cudaError_t launch_seq3_multi<double>(const Grid3 &, const Level3 &, const WarpList3 &, double *,
                                               const double *, cudaStream_t);

cudaError_t prepare_seq3_multi() { return prepare3_t<true>(); }

}  // namespace tmg
