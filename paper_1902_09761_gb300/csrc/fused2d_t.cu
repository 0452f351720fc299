// t = A P^{-1} s of the BiCGStab iteration on 2D grids, s = r - alpha v formed
// on the fly, with the inner products of the omega and next-iteration scalars.
// Kernel template: fused2d.cuh.
#include "fused2d.cuh"

namespace apfc {

template <typename T>
bool launch_fused_t(int m, int Ly, int tile, const OpCoef& c, const ChebStep* w, const cplx<T>* r, const cplx<T>* v,
                    cplx<T>* t_out, const KScal* act, void* partials, cudaStream_t s) {
  LoadS<T> ld{r, v, c.pts};
  EpT<T> ep{t_out, r, v, c.pts};
  // reads r, v; writes t
  return dispatch<T, true>(m, tile, c, w, Ly, ld, ep, act, partials, s, kid_of<T>(KID_FUSED_APINV), 6);
}

template <typename T>
bool launch_fused_merged_t(int m, int Ly, int tile, const OpCoef& c, const ChebStep* w, const cplx<T>* r, const cplx<T>* v,
                           cplx<T>* t_out, const cplx<T>* rhat, const KScal* act, void* partials, cudaStream_t s,
                           const BatchLaunch* bl) {
  LoadS<T> ld{r, v, c.pts};
  EpT5<T> ep{t_out, r, v, rhat, c.pts};
  // reads r, v, rhat; writes t
  return dispatch<T, true>(m, tile, c, w, Ly, ld, ep, act, partials, s, kid_of<T>(KID_FUSED_APINV_T), 8, bl);
}

#define APFC_FUSED_T_INST(T)                                                                                       \
  template bool launch_fused_merged_t<T>(int, int, int, const OpCoef&, const ChebStep*, const cplx<T>*, const cplx<T>*, \
                                         cplx<T>*, const cplx<T>*, const KScal*, void*, cudaStream_t,             \
                                         const BatchLaunch*);                                                     \
  template bool launch_fused_t<T>(int, int, int, const OpCoef&, const ChebStep*, const cplx<T>*, const cplx<T>*,        \
                                  cplx<T>*, const KScal*, void*, cudaStream_t);

APFC_FUSED_T_INST(double)
APFC_FUSED_T_INST(float)

}  // namespace apfc
