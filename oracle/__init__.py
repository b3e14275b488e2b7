"""FP64 CPU oracle for the adjoint-wavelet / blur / channel-gradient hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package may import, call or
execute anything under ``oracle/``; only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.
It shares no code, tables or constants with the CUDA path: filter taps are
derived here from the defining polynomials, extension maps and copy counts are
recomputed from the paper's definitions, and every operator is written as its
plain definition in float64 numpy.

Paper: Folberth & Becker, "Efficient Adjoint Computation for Wavelet and
Convolution Operators" (IEEE SPM Lecture Notes, arXiv 1707.02018).

Modules
  filters    -- Haar / Daubechies / CDF 9/7 filter banks (Sec. I-B, I-C).
  extension  -- extension operators E, copy counts, E^dagger, (E^dagger)^*
                (Sec. I-A, the displayed matrices for E_zpd, E_sym, E_per).
  wavelet    -- one- and multi-level 2D W, W^dagger, W^* (Eq. 2, Eq. 4),
                plus the critically sampled circular transform.
  blur       -- Gaussian PSF, R and R^* (Sec. I, the gradient after Eq. 1).
  conv       -- full convolution and its adjoints (Sec. II, Eq. 5).
  fista      -- objective, power-iteration step size and FISTA (Sec. I-B).
  unrolled   -- unrolled FISTA and its reverse-mode derivative with respect to
                lambda, the PSF width and b (the chain rule of Sec. I).
  layout     -- band sizes and the packed coefficient order.
  cnn        -- the learned warm start x_0 = W^dagger u_hat for FISTA (Sec. I-B
                starts from zero; the 8-layer 3x3 network that computes u_hat
                from b is not in the paper), its loss gradient and Adam.

Every function states the passage it follows.  Functions whose result cannot
be pinned independently say "parity unpinned" in their docstring; at present
every function has at least one independent pin in ``tests/test_oracle_*``.
"""

from . import filters, extension, layout, wavelet, blur, conv, fista, unrolled, cnn  # noqa: F401
