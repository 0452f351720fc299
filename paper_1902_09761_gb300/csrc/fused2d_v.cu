// v = A P^{-1} p of the BiCGStab iteration on 2D grids (unmerged: p formed from
// r, p_old, v_old; merged: r', p' and the previous update formed from r, v, t,
// p, u), with the (rhat, v) inner product.  Kernel template: fused2d.cuh.
#include "fused2d.cuh"

namespace apfc {

// FP32: rhat is read as its packed bf16 copy rh16 (one field transfer instead of two);
// FP64 ignores rh16.
template <typename T>
bool launch_fused_v(int m, int Ly, int tile, const OpCoef& c, const ChebStep* w, const cplx<T>* r, const cplx<T>* p_old,
                    const cplx<T>* v_old, cplx<T>* p_new, cplx<T>* v_new, const cplx<T>* rhat, const uint2* rh16,
                    const KScal* act, void* partials, cudaStream_t s) {
  if (sizeof(T) == 4 && rh16 == nullptr) return false;
  LoadP<T> ld{r, p_old, v_old, p_new, c.pts};
  EpV<T> ep{v_new, rhat, rh16, c.pts};
  // reads r, p_old, v_old (2 fields each) and rhat (FP32: 1, FP64: 2); writes p_new, v_new
  return dispatch<T, true>(m, tile, c, w, Ly, ld, ep, act, partials, s, kid_of<T>(KID_FUSED_APINV),
                           sizeof(T) == 4 ? 11 : 12);
}

template <typename T>
bool launch_fused_merged_v(int m, int Ly, int tile, const OpCoef& c, const ChebStep* w, const cplx<T>* r, const cplx<T>* v,
                           const cplx<T>* t, const cplx<T>* p, cplx<T>* u, cplx<T>* r_new, cplx<T>* p_new,
                           cplx<T>* v_new, const cplx<T>* rhat, const uint2* rh16, const KScal* act, void* partials,
                           cudaStream_t s, const BatchLaunch* bl) {
  if (sizeof(T) == 4 && rh16 == nullptr) return false;
  LoadPR<T> ld{r, v, t, p, u, r_new, p_new, c.pts};
  EpV<T> ep{v_new, rhat, rh16, c.pts};
  // reads r, v, t, p, u (2 fields each) and rhat (FP32: 1, FP64: 2); writes r', p', u, v' (2 each)
  return dispatch<T, true>(m, tile, c, w, Ly, ld, ep, act, partials, s, kid_of<T>(KID_FUSED_APINV),
                           sizeof(T) == 4 ? 19 : 20, bl);
}

#define APFC_FUSED_V_INST(T)                                                                                       \
  template bool launch_fused_merged_v<T>(int, int, int, const OpCoef&, const ChebStep*, const cplx<T>*, const cplx<T>*, \
                                         const cplx<T>*, const cplx<T>*, cplx<T>*, cplx<T>*, cplx<T>*, cplx<T>*,   \
                                         const cplx<T>*, const uint2*, const KScal*, void*, cudaStream_t,         \
                                         const BatchLaunch*);                                                     \
  template bool launch_fused_v<T>(int, int, int, const OpCoef&, const ChebStep*, const cplx<T>*, const cplx<T>*,        \
                                  const cplx<T>*, cplx<T>*, cplx<T>*, const cplx<T>*, const uint2*, const KScal*,  \
                                  void*, cudaStream_t);

APFC_FUSED_V_INST(double)
APFC_FUSED_V_INST(float)

}  // namespace apfc
