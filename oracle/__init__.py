"""FP64 CPU oracle for the BiP-PRISM core-loss map (arxiv 2607.00756).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) imports, links or runs this package; only the tests, the
package's smoke check and the benchmark's CPU-baseline leg do.  It shares no
code with the CUDA path: the two meet only at the seeded inputs of `synth`.

Plain NumPy complex128 / float64, written step by step from the paper:
  physics.py   - interaction constant, wavelength, transmission, Fresnel
                 propagator, one multislice step (Sec. 2.1, Eq. propagator)
  geometry.py  - aperture and detector beams with PRISM subsampling, hex-ring
                 parents, Sibson natural-neighbour weights (Sec. 2.2.3,
                 Eq. nnw, Algorithm 3 build step)
  bip.py       - S1/S2 parent builds, window crop + de-tilt, magnitude-
                 preserving reconstruction, coupling matrix, map
                 (Algorithm 5), the exact dual-matrix map (Algorithm 4) and
                 conventional multislice (Algorithm 1) used as ground truth.
  fp8.py       - the coupling with scaled E4M3 operands (FP64 model)
  mixed.py     - the mixed path's BF16 / FP16 roundings (FP64 model)
  grad.py      - the hand-written reverse pass of the map (Sec. 5)

Parity status: every function is pinned by tests/test_oracle_*.py against
closed forms, invariants, brute force or printed values, except the two
project readings listed as "parity unpinned" in bip.py's header (the absolute
detector-side scale at f > 1 and the hull-boundary weight rule).
"""
