// Split-precision tensor-core form (placeholder until the tcgen05 kernels land).
#include "tc_path.h"

namespace g1g2 {

struct TcPath {
  int nb;
};

int tc_create(TcPath **out, int, int, bool, const cplx *, const cplx *, cudaStream_t) {
  *out = nullptr;
  return G1G2_EUNSUPPORTED;
}

void tc_destroy(TcPath *p) { delete p; }

void tc_rhs(TcPath *, Launcher &, const cplx *, const cplx *, const cplx *, Rk4Stage, cplx *, cplx *, cplx *,
            cplx *, cplx *, cplx *, cplx *, cplx *) {}

}  // namespace g1g2
