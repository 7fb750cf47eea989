"""ctypes declarations of the LES, Poisson and later entry points of
include/gbsw.h (the 2DSW ones are in _native.py)."""
import ctypes as C


class LESParams(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("dx", C.c_double), ("dt", C.c_double),
                ("u_ref", C.c_double), ("z_ref", C.c_double), ("z0", C.c_double), ("cs", C.c_double),
                ("nu", C.c_double), ("alpha", C.c_double), ("beta", C.c_double), ("omega", C.c_double),
                ("tol", C.c_double), ("max_iter", C.c_int), ("check_every", C.c_int)]


class LESStats(C.Structure):
    _fields_ = [("iters", C.c_int), ("status", C.c_int), ("rel_res", C.c_double), ("ms_predictor", C.c_float),
                ("ms_solve", C.c_float), ("ms_guess", C.c_float)]


class LESState(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("u", "v", "w", "p", "fu_old", "fv_old", "fw_old", "gu", "gv", "gw")] + \
               [("step", C.c_int)]


def declare(L, sig):
    vp, ip, dp = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double)
    sig(L, "sw_volume_noalloc", C.c_int,
        [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, vp, vp, vp, vp])
    sig(L, "les_create", C.c_int, [C.POINTER(LESParams), vp, vp, C.POINTER(vp)])
    sig(L, "les_step", C.c_int, [vp, C.c_int, C.POINTER(LESStats)])
    sig(L, "les_get_field", C.c_int, [vp, C.c_int, vp])
    sig(L, "les_set_field", C.c_int, [vp, C.c_int, vp])
    sig(L, "les_get_step", C.c_int, [vp, ip])
    sig(L, "les_set_step", C.c_int, [vp, C.c_int])
    sig(L, "les_set_solver", C.c_int, [vp, C.c_double, C.c_double, C.c_int, C.c_int])
    sig(L, "les_set_check_prediction", C.c_int, [vp, C.c_int])
    sig(L, "les_set_fixed_iterations", C.c_int, [vp, C.c_int])
    sig(L, "les_destroy", None, [vp])
    sp = C.POINTER(C.c_double)
    sig(L, "sw_batch_create", C.c_int, [C.c_int, vp, C.POINTER(sp), C.POINTER(sp), vp, C.POINTER(vp)])
    sig(L, "sw_batch_step", C.c_int, [vp, C.c_int])
    sig(L, "sw_batch_step_separate", C.c_int, [vp, C.c_int])
    sig(L, "sw_batch_volumes", C.c_int, [vp, dp, dp])
    sig(L, "sw_batch_get_state", C.c_int, [vp, C.c_int, vp, vp, vp])
    sig(L, "sw_batch_set_tiling", C.c_int, [vp, C.c_int, C.c_int])
    sig(L, "sw_batch_get_tiling", C.c_int, [vp, ip, ip])
    sig(L, "sw_batch_autotune", C.c_int, [vp, C.c_int, C.c_char_p, ip, ip])
    sig(L, "sw_batch_destroy", None, [vp])
    sig(L, "unet_conv3d", C.c_int, [C.c_int] * 6 + [vp, vp, vp, C.c_int, vp, vp, vp])
    sig(L, "unet_conv3d_bwd_data", C.c_int, [C.c_int] * 6 + [vp, vp, vp, vp, vp])
    sig(L, "unet_conv3d_bwd_weight", C.c_int, [C.c_int] * 6 + [vp, vp, vp, vp, vp])
    sig(L, "unet_glue", C.c_int, [C.c_int] * 6 + [vp, vp, vp, vp, vp])
    sig(L, "unet_head", C.c_int, [C.c_longlong] + [vp] * 9 + [vp])
    sig(L, "unet_num_params", C.c_int, [])
    sig(L, "unet_create", C.c_int, [C.c_ulonglong, vp, C.POINTER(vp)])
    sig(L, "unet_get_params", C.c_int, [vp, vp, C.c_int])
    sig(L, "unet_set_params", C.c_int, [vp, vp, C.c_int])
    sig(L, "unet_forward", C.c_int, [vp, C.c_int, C.c_int, C.c_int, C.c_int, vp, vp])
    sig(L, "unet_infer", C.c_int, [vp, C.c_int, C.c_int, C.c_int, C.c_int, vp, vp])
    sig(L, "les_get_state", C.c_int, [vp, C.POINTER(LESState)])
    sig(L, "les_set_state", C.c_int, [vp, C.POINTER(LESState)])
    sig(L, "unet_gradients", C.c_int, [vp, C.c_int, C.c_int, C.c_int, C.c_int, vp, vp, vp, dp])
    sig(L, "unet_train_step", C.c_int, [vp, C.c_int, C.c_int, C.c_int, C.c_int, vp, vp, C.c_float, dp])
    sig(L, "unet_destroy", None, [vp])
    sig(L, "les_set_warm_start", C.c_int, [vp, vp])
    sig(L, "les_set_warm_start_factor", C.c_int, [vp, C.c_int])
    sig(L, "warm_start_features", C.c_int, [C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, vp, vp, vp, dp, vp])
    sig(L, "warm_start_apply", C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, vp, C.c_double, vp, vp])
    sig(L, "gbsw_selftest_wait", C.c_int, [C.c_int, C.c_longlong])
    sig(L, "gbsw_measure_l2_copy", C.c_int, [C.c_longlong, C.c_int, dp])
    sig(L, "gbsw_debug_bounds", C.c_int, [C.POINTER(C.c_longlong)])
    sig(L, "gbsw_selftest_bounds", C.c_int, [])
    sig(L, "gbsw_selftest_sor_division", C.c_int, [C.c_int, C.POINTER(C.c_ulonglong)])
    sig(L, "poisson_solve", C.c_int, [C.c_int, C.c_int, C.c_int, C.c_double, vp, vp, C.c_double, C.c_double,
                                      C.c_int, C.c_int, vp, ip, dp])
