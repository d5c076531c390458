"""GB300 (sm_103a) implementation of the sketched robust tensor power method of
Wang, Tung, Smola & Anandkumar, "Fast and Guaranteed Tensor Decomposition via Sketching".

The compute path lives in libtsk.so (csrc/*.cu, C ABI in include/tsk.h); this package is its
thin binding.  Entry points: cs_hashes, sketch_tensor, sketch_tensor_planes (with the host
helpers plane_ranges and allreduce_sketches for sketches sharded by planes), sketch_fft,
robust_power_method_sharded (Alg. 1 with the initial vectors split across ranks), sketch_rank1, contract_iuu,
contract_uuu, robust_power_method, decompose_symmetric; asymmetric sketches: sketch_rfft,
contract_ivw, cp_sketch_loss (+ CPSketchLoss autograd function), cp_als_solve, cp_als_step;
many problems: BatchPlan (tsk_batch_create / tsk_batch_run); spectral LDA (Alg. 3):
lda_m2_apply, lda_whiten, lda_whitened_m3, lda_sketch_m3, lda_recover, spectral_lda; order-p
symmetric sketches: cs_hashes_p, sketch_tensor_p, contract_p, robust_power_method_p; roof
micro-kernels: peak_launch, peak_work.
"""
from .api import (cs_hashes, sketch_tensor, sketch_tensor_planes, plane_ranges,  # noqa: F401
                  allreduce_sketches, select_first_max, robust_power_method_sharded,
                  sketch_fft, sketch_rank1,
                  contract_iuu, contract_uuu, robust_power_method, decompose_symmetric,
                  robust_power_method_launches, robust_power_method_asym, ctx_status, check_status, sketch_rfft,
                  contract_ivw, cp_sketch_loss, CPSketchLoss, cp_loss, cp_als_solve, cp_als_step,
                  BatchPlan, lda_m2_apply, lda_whiten, lda_whitened_m3, lda_sketch_m3,
                  lda_recover, spectral_lda, cs_hashes_p, sketch_tensor_p, contract_p,
                  robust_power_method_p, robust_power_method_p_launches, peak_launch, peak_work,
                  PEAK_FMA, PEAK_SMEM, PEAK_ATOMS)
from ._lib import TskError, LIB_PATH, load as load_library  # noqa: F401
