// Stencil kernels instantiated for the StoreDF storage kind (one translation
// unit per kind so that the kinds compile in parallel).
#include "stencil_kernels.cuh"

namespace bcg {

BCG_DSLASH_KIND_DECL(dslash_df) {
  if (R & DSLASH_TC) {
    if (dslash_tc_supported(g, N))
      return dslash_df_tc(epi, links, in, out, c1, c2, m2, g, out_parity, N, gate, s);
    R = (R & ~DSLASH_TC) | DSLASH_ASYNC;  // other widths: the cp.async kernel
  }
  return dslash_kind<StoreDF>(R, epi, links, in, out, c1, c2, m2, g, out_parity, N, gate, s);
}

}  // namespace bcg
