"""FP64 CPU oracle for the Snake-NeRF per-tile training step.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` call it.  It shares no code with the CUDA library; the
only common module is ``synth`` (seeded input generators, none of the
method's arithmetic).

Each module restates one step of the method in plain numpy, in the order the
paper (and the works it defers to) defines it:

* ``philox``   - counter-based RNG (Salmon et al. 2011) used for stratified
                 jitter and parameter initialisation.
* ``camera``   - localisation of a pixel with an affine or cubic rational
                 (RPC-like) camera and the ray through z_max / z_min
                 (Sec. 3 and Sec. 4.6: rays are computed when needed).
* ``sampler``  - ray/box clipping, 2x2-window acceptance (Sec. 4.4) and the
                 segmented sampler (Sec. 4.5).
* ``hashgrid`` - multiresolution hash encoding (Sec. 4.1, NGP).
* ``mlp``      - local density MLP and shared colour MLP (Sec. 4.1).
* ``render``   - front-to-back volume rendering (NeRF Eq. 3, Sec. 4.5).
* ``adam``     - Adam as used by I-NGP (Sec. 4.6).
* ``step``     - one training step and one render call put together.
* ``targets``  - FP64 ray/heightfield renderer for the synthetic target images.

Floating point is FP64 throughout, except where a float decides an integer
(segment bounds, sample positions, grid cells, samples per segment): those
decisions are defined as a fixed sequence of IEEE binary32 operations and the
oracle evaluates that sequence with numpy float32 (no fused multiply-add), so
the CUDA path can be compared bit for bit.

Pins: every function here is checked by ``tests/test_oracle_*.py`` against
closed forms, invariants, brute force or finite differences.  The choices the
paper leaves open (samples per segment, bin convention, MLP details, loss,
Adam hyper-parameters) are pinned only by those invariants; they are listed
as readings, not as the paper's own statements.
"""
