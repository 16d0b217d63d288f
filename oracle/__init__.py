"""FP64 CPU oracle for the in-plane self-gravity of an infinitesimally thin disk.

TEST INFRASTRUCTURE ONLY. Nothing in the product path (the CUDA library and its
Python binding) imports, links or executes this package; only the tests, the
smoke check and the CPU-baseline leg of the benchmark do. It shares no code,
headers, tables or constants with the CUDA path.

What it computes (Tseng, Shang & Yen, Section 2):

* ``kernels``  -- the closed-form cell integrals K^{x,0}, K^{x,x}, K^{x,y} and
  the y-family of the force kernel at z = 0 (Section 2, the antiderivative list
  and the coincident-line modification), and the nine off-plane integrals with
  the arctan terms, vectorised in numpy.
* ``direct``   -- the plain O(N_t * N_s) sum F = G sum_i [sigma0_i K^{.,0}_i +
  deltax_i K^{.,x}_i + deltay_i K^{.,y}_i] over arbitrary rectangular source
  cells (Eq. eqnXforce2 with the order-1 Taylor reconstruction of Eq. eqnGamma),
  written in plain C with OpenMP over targets.
* ``fftconv``  -- the uniform-grid route: the same sum as a zero-padded
  convolution evaluated with numpy's FFT (a library primitive), as the paper's
  introduction and conclusion describe for uniform grids.
* ``amr``      -- leaf enumeration of a nested-patch hierarchy (Section 3,
  Fig. 1) and of a zone-by-zone hierarchy (Table 10, Section 4), and the AMR
  force as the flattened leaf-pair sum.
* ``potential``-- the mid-plane potential Phi = -G integral sigma / r (Section 2,
  the singular kernel integral) with the order-1 reconstruction: closed-form
  cell integrals, the plain C sum and the FFT route.
* ``disks``    -- closed-form forces of the D_2 disk (Section 3) and the Kuzmin
  disk, the D_2 mid-plane potential, used as pins.
* ``norms``    -- the L1, L2, Linf error norms of Section 3 and the AMR norms of
  Section 4.

Every floating-point step is FP64.
"""
