"""GB300-native k-center farthest-point path (McClintock & Wirth, arXiv 1604.03228).

The CUDA library (``csrc/``, C ABI in ``include/kcenter.h``) does the work;
``binding`` marshals arguments to it.  ``inputs`` draws seeded synthetic
point sets shaped like the paper's workloads.
"""
from .binding import (KC_ASYNC, KC_AUTOTUNE, BatchPlan, kc_batch_plan_create, kc_batch_plan_destroy,  # noqa: F401
                      kc_batch_plan_info, kc_batch_plan_run, kc_batch_plan_wait, KC_ERR_ARG, KC_ERR_CUDA, KC_ERR_NONFINITE, KC_ERR_OOM,  # noqa: F401
                      KC_ERR_RANGE, KC_ERR_TIMEOUT, KC_F32, KC_I32, KC_OK, KC_SWEEP_BF16, KC_SWEEP_F32,
                      KC_SWEEP_FP8, KC_SWEEP_FP16, KC_TEST_WITHHOLD, GonResult, KCError,
                      RadiusResult, kc_eim, kc_gonzalez, kc_gonzalez_batch, kc_gonzalez_noalloc, kc_mrg_rounds,
                      kc_counters, kc_last_fp32_radius, kc_launch_count, kc_mrg, kc_radius, kc_read_sweep, kc_release, kc_sync,
                      kc_trace_enable, kc_trace_read, kc_version, library_path, load)
