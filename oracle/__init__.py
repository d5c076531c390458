"""FP64 CPU oracle for the sketched robust tensor power method of
Wang, Tung, Smola & Anandkumar, "Fast and Guaranteed Tensor Decomposition via Sketching"
(NIPS 2015).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline /
reference legs may import this package.  It shares no code with the CUDA path and never
imports it; both sides read inputs from the seeded generators in `synth`.

Modules (each function cites the passage it follows):
  hashing  -- hash family h, complex Rademacher sigma (Sec. 3.3, Prop. 2)
  conv     -- circular convolution / correlation, direct and FFT engines (Prop. 1, App. F)
  sketch   -- count sketches and tensor sketches by definition (Eq. 1, Eq. 4, Eq. 7, App. B)
  contract -- exact and sketched T(I,u,u), T(u,u,u), T(I,v,w) (Sec. 3.2, App. B)
  rtpm     -- plain and sketched robust tensor power method (Sec. 2, Alg. 1)
  cp       -- sketched CP loss and gradient, sketched ALS update (Alg. 2, Eq. 15)
  lda      -- spectral LDA moments, whitening, whitened M3, recovery (App. D, Alg. 3)
  orderp   -- order-p symmetric sketches, their contractions and Alg. 1 for p >= 3 (Sec. 3.3)

Parity pins: every function is checked in tests/test_oracle_pins.py against facts fixed by
the paper or by mathematics (collision-free exactness, Prop. 1, Lemma 1 unbiasedness and
variance bound, planted-component recovery, invariants); see that file.
"""
from . import hashing, conv, sketch, contract, rtpm  # noqa: F401
from .hashing import cs_hashes, sigma_of, xi_of  # noqa: F401
from .sketch import (count_sketch, count_sketch_asym, sketch_tensor_sym,  # noqa: F401
                     sketch_tensor_sym_sorted, sketch_truncated_sym, sketch_tensor_asym,
                     sketch_rank1_sym, sketch_rank1_asym, recover_entry_sym)
from .contract import (exact_iuu, exact_uuu, exact_ivw, contract_iuu, contract_uuu,  # noqa: F401
                       contract_iuu_def, contract_uuu_def, contract_ivw_asym)
from .rtpm import (median, median_rows, rtpm_sketched, rtpm_sketched_asym, rtpm_exact,  # noqa: F401
                   power_step_sketched,
                   eigenvalue_sketched, deflate_sketches, NonFiniteError)
from . import cp  # noqa: F401,E402
from .cp import (cp_sketch_loss, cp_sketch_grad, cp_exact_loss, contract_ivw_mode,  # noqa: F401,E402
                 als_sketched_columns, als_solve)
from . import lda  # noqa: F401,E402
from . import orderp  # noqa: F401,E402
