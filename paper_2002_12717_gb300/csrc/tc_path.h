// Split-precision tensor-core form of the G1-G2 right-hand side (internal).
#pragma once

#include "g1g2_internal.h"

namespace g1g2 {

struct TcPath;

// Build the tensor-core path for one context. hw: w (complex, [(ij),(kl)]),
// hsrc: source-term interaction (w^- for SOA in a spin-orbital basis, else w).
// sliced: BF16-slice operands with an exact leading product instead of TF32 hi/lo.
// bosons: nbar = 1 + n (instead of 1 - n) and the sign of the particle-hole quasi-Hamiltonian.
int tc_create(TcPath **out, int nb, int se, bool restricted, bool sliced, bool bosons, const cplx *hw, const cplx *hsrc,
              cudaStream_t stream);
void tc_destroy(TcPath *p);

// Refresh the FP32 copy of the G2 state (after init / set_state).
void tc_load_state(TcPath *p, Launcher &L, const cplx *G);
// G1G2_ETIMEOUT when a tensor-core kernel gave up on a barrier (synchronises the stream).
int tc_error(TcPath *p, cudaStream_t stream);
// Launch a wait on a barrier nothing arrives on, bounded by limit_ns:
// G1G2_ETIMEOUT when the wait gave up and reported it (the expected result).
int tc_wait_selftest(unsigned long long limit_ns, cudaStream_t stream);

// One right-hand side (hhf already built from n_in): collision integral and
// G1 update, then the G2 contractions and the assembly with the RK4 update.
void tc_rhs(TcPath *p, Launcher &L, const cplx *n_in, const cplx *G_in, const cplx *hhf, Rk4Stage st,
            cplx *ny, cplx *nys, cplx *nacc, cplx *nk, cplx *Gy, cplx *Gys, cplx *Gacc, cplx *Gk);

}  // namespace g1g2
