"""CPU oracle for the block-filtered exchange-correlation quadrature.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 restatement of
what the method computes, written from the paper's equations.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference leg may
import it.  It shares no code with the GPU library (``paper_2605_10363_gb300``)
and imports nothing from it; the only module both use is ``synth`` (seeded
inputs, no method arithmetic).

Modules
  basis   contracted Cartesian Gaussians, values and gradients   (App. A)
  grid    atom-centred grid, Becke partition, Morton order, blocks (App. A, App. B Eq. morton_code)
  screen  block summaries, retention, executed pairs, Alg. 1       (Sec. III-B-3, III-C-1, App. D)
  xc      LDA exchange and PBE-form GGA energy densities           (Sec. II-A; functional forms in xc.py)
  exc     dense and screened rho / E_xc / V_xc                      (Sec. II-A Eqs. exc_quadrature..fxc_matrix_form,
                                                                      Sec. III-C Eq. executed_block_output)
  mlp     2-64-64-2 surrogate forward/backward in FP64              (no counterpart in the paper)

Parity pins (each checked by ``tests/test_oracle_*.py`` against something other
than the oracle itself) are listed in each module's header.  Parity unpinned:
the absolute accuracy of the quadrature grid (only its exactness on
polynomials and Gaussians is pinned).
"""
