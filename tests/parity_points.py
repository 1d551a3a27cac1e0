"""The (beta, Delta, n_max, D_cut, n_steps) points of the GPU parity tests.

Kept in one place so that tests/test_oracle_conditioning.py can check, on the
CPU, that each point is well conditioned: a relative perturbation of the
input tensor at the level of the arithmetic used must move the oracle's
ln Z / N by far less than the parity tolerance.  Otherwise the FP64 answer
itself is not fixed to that tolerance and no implementation could match it.
"""

# FP64 form, |d lnZ/N| <= 1e-10.
FP64_SHAPES = [
    (1.6, 0.3, 3, 13, 14),    # odd D_cut: ragged tiles everywhere
    (0.7, 0.8, 4, 24, 12),
    (1.2, 0.1, 1, 9, 10),     # D_cut = D_h^2 at the first step
    (0.5, 0.5, 0, 4, 6),      # D0 = 1: the trivial tensor
    (1.0, 0.5, 2, 1, 5),      # D_cut = 1
    (1.0, 0.5, 2, 16, 0),     # no step: closing trace of T0
    (1.0, 0.5, 2, 12, 10),    # mirror-image environments: eps_1 = eps_2 at every step
]

# Split BF16 form, |d lnZ/N| <= 1e-9.
SPLIT_SHAPES = [
    (1.0, 0.5, 2, 16, 20), (1.6, 0.3, 4, 16, 25), (0.7, 0.8, 4, 24, 14), (1.2, 0.1, 3, 13, 12),
    (2.0, 0.9, 4, 16, 25), (1.0, 0.5, 2, 13, 10), (0.9, 0.6, 3, 20, 24),
]

# Batched runner: eight points of two tensor classes; the first three are also
# compared with the oracle.
BATCH_STEPS = 10
BATCH = [(b, d, 2 + i % 2, dc, BATCH_STEPS) for i, (b, d, dc) in enumerate(
    [(1.0, 0.5, 13), (1.6, 0.3, 16), (0.7, 0.8, 12), (1.2, 0.1, 16), (0.9, 0.6, 12),
     (2.0, 0.9, 16), (1.1, 0.4, 9), (0.8, 0.2, 12)])]
BATCH_ORACLE = BATCH[:3]

# Ill-conditioned counter-example: after about ten steps the cut at D_cut = 12
# amplifies any perturbation roughly a thousandfold per step, so 1e-15 input
# noise moves the oracle's own ln Z / N by ~1e-7 at 14 steps (and 1e-10 noise,
# the split form's level, by ~1e-8 already at 10 steps; D_cut = 13 is benign).
ILL_CONDITIONED = (1.0, 0.5, 2, 12, 14)

# The q != 2 couplings (cos(q theta)), (beta, Delta, n_max, D_cut, n_steps, q).
Q_SHAPES = [(1.1, 0.5, 3, 16, 12, 3), (0.9, 0.7, 3, 13, 10, 4), (1.2, 0.4, 2, 12, 10, 1)]

# Ordered phase (T = 0.55 at Delta = 0.32): the kept U(1) window drifts away
# from charge 0 late in the run (an exact +-q pair split at the cut keeps +q,
# and fusing doubles an off-centre window every two steps), so the signed
# label sums of the block-sparse products leave [-64, 63] (by step 25 at
# D_cut = 12, step 29 at D_cut = 24) while their span stays small.
DRIFT_SHAPES = [(1 / 0.55, 0.32, 4, 12, 30), (1 / 0.55, 0.32, 4, 24, 30)]
