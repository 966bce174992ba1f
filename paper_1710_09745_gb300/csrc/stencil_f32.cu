// Stencil kernels instantiated for the StoreF32 storage kind (one translation
// unit per kind so that the kinds compile in parallel).
#include "stencil_kernels.cuh"

namespace bcg {

BCG_DSLASH_KIND_DECL(dslash_f32) {
  return dslash_kind<StoreF32>(R, epi, links, in, out, c1, c2, m2, g, out_parity, N, gate, s);
}

}  // namespace bcg
