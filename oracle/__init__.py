"""FP64 CPU oracle for the UMAP-style neighbour-embedding hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) imports, links or executes anything under ``oracle/``;
only the tests, the smoke check of ``__graft_entry__`` and the CPU-baseline leg
of ``bench.py`` do.  The oracle shares no code with the CUDA path.

The paper (mlx-vis, Section 2.3, and the UMAP method it cites in Section 1)
names the method's stages but does not print their equations, so each stage
below follows the published UMAP construction, in plain NumPy/SciPy, in FP64:

* ``knn``            exact brute-force k-NN (Section 2.2 computes distances by
                     the expansion |a|^2+|b|^2-2a.b; here that expansion only
                     shortlists candidates, whose squared distances are then
                     recomputed directly as sum (x-y)^2).
* ``fuzzy``          per-point rho, sigma by bisection so that the row weight
                     sum equals log2 k; directed weights; fuzzy union; CSR
                     sorted by (head, tail); integer epoch schedule words.
* ``curve``          the a, b fit of the output kernel 1/(1+a x^(2b)) by
                     Gauss-Newton (Section 2.3).
* ``philox``         Philox4x32-10 (Salmon et al., SC'11) in NumPy integers.
* ``sgd``            uniform initialisation, the synchronous SGD epoch
                     (attraction along active edges, repulsion from negative
                     samples, clip to +-4) and the full fit (Section 3,
                     500 epochs; Section 3.2, the optimisation loop).
* ``metrics``        k-NN preservation and trustworthiness (Section 3.2).
* ``spectral``       the spectral initial layout: the leading non-trivial
                     eigenvectors of the normalised fuzzy-graph adjacency.
* ``render``         the circle-splatting renderer (Section 2.4): linear
                     falloff splats, premultiplied accumulation, resolve.
* ``pca``            PCA preprocessing to pca_dim (Section 3): covariance,
                     leading eigenvectors, projection.
* ``nndescent``      the approximate k-NN graph by NNDescent (Section 2.2):
                     random start, neighbours-of-neighbours refinement,
                     early stop at update rate 0.015.
* ``mlp``            FP64 forward/backward of the learned 50-256-256-2 embedder
                     with BF16 rounding emulated where the CUDA path rounds.

Parity status: every function is pinned by the ``-m "not gpu"`` tests against
something other than itself (library routines, closed forms, finite
differences, invariants or published constants).  ``sgd.fit`` is a chaotic
iteration and is pinned only through its parts and through statistics.
"""
from . import knn, fuzzy, curve, philox, sgd, metrics, mlp, spectral, render, pca, nndescent  # noqa: F401
