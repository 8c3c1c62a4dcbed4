"""Plain CPU FP64 oracle for hybrid DH^2 compression (Boerm & Boerst, arXiv 1809.04384).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
link this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA library (``paper_1809_04384_gb300``); the only common
module is ``synth`` (seeded input generators, no method arithmetic).

The oracle follows the paper step by step, in the paper's order and notation,
with numpy (FP64, complex128) and ``numpy.linalg`` QR/SVD as library steps:

* ``geometry``      - kernel g (Eq. 1), Galerkin entries (Eq. 2), quadrature,
                      dense matrix G (the ground truth).
* ``structure``     - cluster tree (Def. "cluster tree"), bounding boxes,
                      directions (Def. "directions", Remark "construction of
                      directions"), son map sd, c_ts, block tree (Def. "block
                      tree"), row/col sets.
* ``interp``        - directional Chebyshev interpolation: leaf bases V_tc,
                      transfer matrices E_t'c (Eq. nested_apx), couplings S_b
                      (Eq. matrix_apx), and the interpolated DH^2 matvec.
* ``recompress``    - Section 3.2: basis weights R (Eq. basis_weights_def),
                      total weights Z-hat (Eq. recomp_weight_full), truncation
                      to Q/F/C, projection of couplings (Lemma "Projections"),
                      and the recompressed DH^2 matvec.
* ``dense_compress``- Section 3.1 on an explicitly expanded matrix (tiny meshes).
* ``learned``       - the learned order/rank model: features, interpolation-error
                      labels, MLP forward/backward with BF16 weights, Adam.
* ``double_layer``  - the double-layer potential (Section 5's second operator):
                      kernel and dense Galerkin matrix, the ground truth of the next
                      operator the GPU path takes on.

Parity status per function is stated in each module header; the one value
with no pin (the distance of the DH^2 approximation from the dense matrix,
which is interpolation error) is marked "parity unpinned" there.
"""
