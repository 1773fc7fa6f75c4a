"""Plain FP64 CPU oracle for the PSMS hot path (Finkenrath, Knechtli, Leder,
"Fermions as Global Correction: the QCD Case", arXiv:1204.1306).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product library never calls it and shares no code with it.

Every routine here is a direct, slow restatement of the paper's definitions:
full-lattice numpy arrays in the canonical lexicographic layout
``[x0][x1][x2][x3]`` (x3 fastest, mu=0 is time), explicit 4x4 gamma matrices,
no even-odd split and no half-spinor projection.

Modules
-------
philox     Philox-4x64-10 counter-based generator and the draw map.
lattice    geometry: shifts, parity, domain blocks, black/white colouring,
           active links (Sec. 3), the projector P (Sec. 4.4).
gamma      Euclidean gamma matrices in the chiral basis.
gauge      link generator, plaquette action (Eq. (Sw)), staples,
           Cabibbo-Marinari heatbath / overrelaxation (Sec. 6).
dirac      Wilson-Dirac operator (Eq. (Dw)), Dirichlet block operators,
           black/white hopping pieces (Eq. (domdec)), dense assembly.
linalg     CGNR solver and a partial-pivot LU for log|det|.
estimator  stochastic determinant-ratio estimates (Eqs. (stacc), (staccN),
           (gfparam), (detschur), (inverseschur)).
filter     accept/reject decisions and one hierarchical filter step
           (Eq. (hierarchy), Sec. 3 and App. A).
mlp        learned delayed-acceptance level: domain features and an FP64
           MLP forward/backward.
gaugefix   relative gauge fixing of a pair of fields (Sec. 4.2, App. B).
hyp        one level of HYP smearing and the block HYP plaquette action of
           the parametrised levels (App. C, Sec. 5).
params     coefficients of the parametrised levels (App. C, Eq. (paramsi)).
recursive  recursive domain decomposition (Eq. (ddrec)): nested blocks, the
           Schur complements of the outer blocks and their stochastic
           estimate, and the filter step with one level of recursion
           (Eq. (4step)).

Pins: functions are checked in ``tests/test_oracle_*.py`` against closed forms,
library routines and numbers printed in the paper (``tests/golden``).
"""
