// Stencil kernels instantiated for the StoreH16 storage kind (one translation
// unit per kind so that the kinds compile in parallel).
#include "stencil_kernels.cuh"

namespace bcg {

BCG_DSLASH_KIND_DECL(dslash_h16) {
  if (R & DSLASH_TC) {
    if (dslash_tc16_supported(N) && !(R & DSLASH_RECON))
      return dslash_tc16(FK_H16, epi, links, in, out, c1, c2, m2, g, out_parity, N, gate, s);
    R &= ~DSLASH_TC;  // other widths: the plain kernel
  }
  return dslash_kind<StoreH16>(R, epi, links, in, out, c1, c2, m2, g, out_parity, N, gate, s);
}

}  // namespace bcg
