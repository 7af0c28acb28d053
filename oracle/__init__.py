"""Plain FP64 CPU oracle for boundary-MPS row absorption with rSVD compression.

TEST INFRASTRUCTURE ONLY. Nothing on the product path imports, calls or links
this package: only the tests, ``__graft_entry__.smoke()`` (which checks one
small GPU run against it) and the CPU-baseline leg of ``bench.py`` use it.

It restates, slowly and in double precision, what the GPU path computes:

* ``philox``   - the Philox4x64-10 counter-based generator and the Box-Muller
                 Gaussian sketch Omega (paper Sec. IV: Omega is Gaussian).
* ``network``  - the PEPS-PEPO-PEPS sandwich (Sec. II, Fig. 1), brute-force
                 state vectors for small lattices and an independent exact
                 column-wise contraction.
* ``boundary`` - the boundary-MPS environment approximation (Sec. II) with
                 rSVD compression (Sec. IV, Halko et al. Example 1.6) and the
                 CBE variational fit whose A*Omega follows Fig. 5 (n_fit passes,
                 re-canonicalised left to right between them).
* ``symmetric`` - the U(1) x U(1) block-sparse mode (Sec. III quantum-number
                 slicing, Sec. V symmetric Hubbard runs): the zip-up with a
                 sector-wise rSVD and one global truncation, and the CBE fit
                 with a sector-wise CBE rSVD and a sector-wise SVD of the
                 fitted tensor, on the dense applications of ``boundary``.
* ``blocksparse`` - the four site maps (Theta_c, its transpose, the fit's
                 right-environment map and its transpose) by charge blocks
                 (Sec. III quantum-number slices): one task per output block of
                 each of their three contractions, with the task lists.

It shares no code with the CUDA path; the only common module is the seeded
input generator ``synth`` (data, no method arithmetic).
"""
