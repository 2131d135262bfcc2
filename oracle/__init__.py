"""FP64 CPU oracle for the subsampled randomized (H-)Tucker decomposition.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA library (no kernels, headers, helpers or constant
tables); the only thing both sides share is the seeded input generators in
``synth/``, which hold none of the method's arithmetic.

Layout of the oracle, each function citing the passage of arXiv 2603.21379
("A practical mode-parallel implementation of the (H-)Tucker decomposition via
randomization") that it follows:

* ``rng``      - the counter-based random streams the method draws: fiber
                 indices sampled uniformly without repetition (Sec. 3.1) and
                 the Gaussian test matrices Omega_k (Sec. 3.1, Alg. 1).
* ``tucker``   - unfoldings, TTM and multi-TTM (Sec. 2.2), Sub-R-HOSVD
                 (Alg. 1), reconstruction and relative error.
* ``htucker``  - dimension tree (Sec. 4, Def. 4.1), Sub-R-RtL-HT (Alg. 2),
                 transfer tensors (Eqs. 4.1/4.2), H-Tucker reconstruction.
* ``brute``    - deterministic T-HOSVD (Sec. 3) and RtL-HT (Sec. 4) by full
                 SVDs, used only to pin the randomized oracle on tiny inputs.
* ``tucker_grad`` - gradients of the Tucker misfit 1/2 ||X - G x_k U_k||^2 and
                 the adjoint of the core projection (Sec. 3 format, Alg. 1
                 core step); the differentiable extension, not in the paper.
* ``fp8``      - float8 (E4M3) storage of X with one power-of-two scale per
                 slab of the last two modes (the FP8 form; not in the paper).
* ``rhkron``   - randomized HOSVD with Kronecker-structured Gaussian test
                 matrices, the rHKron comparison method of Sec. 3.3 (its
                 reduced core factored mode by mode).

Precision: every floating-point step runs in float64 (the paper's NumPy
implementation does not state a precision; float64 is NumPy's default).
"""

from . import rng, tucker, htucker, brute, tucker_grad  # noqa: F401
