"""Plain CPU oracle for the blockwise 2-D Chen-approximation DCT pipeline.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It
shares no code, tables or helpers with the CUDA library; the only common
dependency is the seeded input generator ``paper_2207_11638_gb300.synth``,
which holds none of the method's arithmetic.

Everything here is written from the paper ("DCT Approximations Based on
Chen's Factorization", arXiv 2207.11638) as explicit matrix definitions and
explicit matrix products, in exact integers (int64 / Python ints /
fractions) or float64:

* ``matrices``  -- the factor matrices of Eqs. 1-3, the parametric map T_C
  (Sec. 3), sign/round parameter vectors, T~8 and T^8 (Eqs. 4-5), their
  inverses (Eqs. 6-7), the diagonal scale S (Sec. 3.1), the JAM recursion for
  N = 16, 32 (Sec. 6.1) and the exact DCT-II / DCT-IV (Sec. 2).
* ``pipeline``  -- the JPEG-like experiment of Sec. 5.1: per-block forward
  transform, zig-zag zonal retention of r coefficients, inverse transform and
  PSNR, for the approximations and for the exact DCT.
* ``metrics``   -- deviation from diagonality (Sec. 3.1), total error energy
  and unified coding gain (Sec. 4.1), additive complexity (Tables 2 and 4),
  and the SSIM index the experiment of Sec. 5.1 reports.
* ``rd``        -- the exhaustive rate-distortion quadtree search over 32 x 32
  regions (transform sizes 32 / 16 / 8, as in the codec of Sec. 6.2).
* ``cnn``       -- the learned size selector that proposes the quadtree
  instead: forward, backward, loss and Adam in float64 with the GPU's
  bfloat16 rounding points.

Parity status per function is stated in each function's docstring: every
function is pinned by at least one ``-m "not gpu"`` test except the coding
gain of the approximations (the paper's Fig. 3 is not available), which is
"parity unpinned".
"""
