"""ctypes binding of libpgb (include/pgb.h): one Python function per C entry
point, with the same name, doing argument marshalling only.  Device arrays are
passed as torch CUDA tensors (their data_ptr is handed to the library);
host arrays as numpy arrays.  A negative status raises PgbError, except
PGB_ENOCONV from pgb_solve, which is returned with the stats."""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpgb.so")

PGB_OK, PGB_EINVAL, PGB_ENOMEM, PGB_ECUDA, PGB_ENOCONV, PGB_ETIMEOUT, PGB_ESTATE = 0, -1, -2, -3, -4, -5, -6
PGB_ECOLL = -7
PGB_DIELECTRIC, PGB_SET_CHARGE, PGB_SET_POTENTIAL = 0, 1, 2
PGB_FP32, PGB_FP64, PGB_FP32_REFINE, PGB_FP64_DS = 0, 1, 2, 3

c_i32, c_i64, c_dbl, c_vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p


class pgb_params(ctypes.Structure):
    _fields_ = [("K", c_i32), ("K_near", c_i32), ("n_edge", c_i32), ("P", c_i32), ("theta", c_dbl),
                ("leaf_size", c_i32), ("group_size", c_i32), ("p2p_item", c_i32), ("m2p_item", c_i32),
                ("precond", c_i32), ("graphs", c_i32), ("lanes", c_i32),
                ("overlap", c_i32), ("batch", c_i32), ("residual", c_i32)]


class pgb_solve_stats(ctypes.Structure):
    _fields_ = [("iterations", c_i32), ("outer_steps", c_i32), ("matvecs", c_i32), ("matvecs_fp64", c_i32),
                ("rel_residual", c_dbl)]


class pgb_energies(ctypes.Structure):
    _fields_ = [("coulomb", c_dbl), ("solvation", c_dbl), ("surface", c_dbl), ("total", c_dbl)]


class pgb_tree_info(ctypes.Structure):
    _fields_ = [(n, c_i64) for n in ("n_panels", "n_unknowns", "n_nodes", "n_leaves", "n_groups", "n_near",
                                     "n_far", "p2p_pairs", "p2p_laplace_pairs", "m2p_pairs", "m2p_laplace_pairs",
                                     "n_corrections", "n_p2p_items", "n_m2p_items")]


N_STAGES = 14
STAGES = ("sources", "upward", "p2p", "m2p", "assemble", "krylov", "tree", "energy", "rhs",
          "sources_fp64", "upward_fp64", "p2p_fp64", "m2p_fp64", "assemble_fp64")


class pgb_stage_times(ctypes.Structure):
    _fields_ = [("ms", c_dbl * N_STAGES), ("calls", c_i64 * N_STAGES), ("kernel_launches", c_i64),
                ("host_launches", c_i64)]


class PgbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"pgb error {code}: {msg}")
        self.code = code


_lib = None

_SIGS = {
    "pgb_create": (c_i32, [ctypes.POINTER(c_vp), ctypes.POINTER(pgb_params), c_vp]),
    "pgb_destroy": (c_i32, [c_vp]),
    "pgb_last_error": (ctypes.c_char_p, [c_vp]),
    "pgb_default_params": (c_i32, [ctypes.POINTER(pgb_params)]),
    "pgb_mesh_load": (c_i32, [c_vp, c_i32, c_vp, c_i64, c_vp, c_i64, c_dbl, c_vp, c_vp, c_i64, c_dbl,
                              ctypes.POINTER(c_i32)]),
    "pgb_set_solvent": (c_i32, [c_vp, c_dbl, c_dbl]),
    "pgb_set_charges": (c_i32, [c_vp, c_i32, c_vp, c_i64]),
    "pgb_set_bc": (c_i32, [c_vp, c_i32, c_dbl]),
    "pgb_autotune": (c_i32, [c_vp, c_vp, c_i32, c_vp, c_i32, c_vp, c_i32, c_i32, c_dbl, c_dbl,
                             ctypes.POINTER(pgb_params), c_vp]),
    "pgb_set_pose": (c_i32, [c_vp, c_i32, c_vp, c_vp]),
    "pgb_set_region": (c_i32, [c_vp, c_i32, c_i32, c_dbl]),
    "pgb_tree_build": (c_i32, [c_vp]),
    "pgb_tree_reset": (c_i32, [c_vp]),
    "pgb_tree_refresh": (c_i32, [c_vp]),
    "pgb_tree_stats": (c_i32, [c_vp, ctypes.POINTER(pgb_tree_info)]),
    "pgb_num_unknowns": (c_i32, [c_vp, ctypes.POINTER(c_i64)]),
    "pgb_matvec": (c_i32, [c_vp, c_vp, c_vp, c_i32]),
    "pgb_rhs": (c_i32, [c_vp, c_vp]),
    "pgb_solve": (c_i32, [c_vp, c_i32, c_dbl, c_i32, c_i32, c_vp, ctypes.POINTER(pgb_solve_stats)]),
    "pgb_energy": (c_i32, [c_vp, c_vp, ctypes.POINTER(pgb_energies), c_vp]),
    "pgb_solve_batch": (c_i32, [c_vp, c_i32, c_vp, c_vp, c_i64, c_i32, c_dbl, c_i32, c_i32, c_vp, c_vp]),
    "pgb_solve_poses": (c_i32, [c_vp, c_i32, c_vp, c_i32, c_vp, c_vp, c_i64, c_i32, c_dbl, c_i32, c_i32, c_vp,
                                c_vp]),
    "pgb_grad": (c_i32, [c_vp, c_vp, c_i32, c_dbl, c_i32, c_i32, c_vp, c_vp, c_vp, ctypes.POINTER(pgb_solve_stats)]),
    "pgb_matvec_transpose": (c_i32, [c_vp, c_vp, c_vp, c_i32]),
    "pgb_tree_export": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "pgb_timing": (c_i32, [c_vp, c_i32, ctypes.POINTER(pgb_stage_times)]),
    "pgb_energy_noalloc": (c_i32, [c_vp, c_vp, ctypes.POINTER(pgb_energies)]),
    "pgb_math_check": (c_i32, [c_vp, c_i64, c_vp]),
    "pgb_alloc_count": (c_i32, [ctypes.POINTER(c_i64)]),
    "pgb_far_table": (c_i32, [c_i32, c_dbl, c_vp, c_i64]),
    "pgb_orientation_landscape": (c_i32, [c_vp, c_i32, c_i32, c_dbl, c_vp]),
    "pgb_shard_partition": (c_i32, [c_vp, c_i64, c_i32, c_vp]),
    "pgb_shard_rows": (c_i32, [c_vp, c_i32, c_vp]),
    "pgb_to_sharded": (c_i32, [c_vp, c_vp, c_vp, c_i32]),
    "pgb_matvec_shard": (c_i32, [c_vp, c_i32, c_i32, c_vp, c_vp, c_i32]),
    "pgb_solve_shard": (c_i32, [c_vp, c_i32, c_i32, c_vp, c_vp, c_vp, c_vp, c_i32, c_dbl, c_i32, c_i32, c_vp,
                                ctypes.POINTER(pgb_solve_stats)]),
}


def lib():
    """The loaded CDLL; raises if the library has not been built (there is no
    fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with python -m paper_1506_03745_gb300.build")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(ctx, st, allow=()):
    if st < 0 and st not in allow:
        msg = lib().pgb_last_error(ctx).decode() if ctx else ""
        raise PgbError(st, msg)
    return st


def _dptr(t, dtype_name, n=None):
    """Device pointer of a contiguous CUDA tensor (torch), checked."""
    if not (hasattr(t, "is_cuda") and t.is_cuda and t.is_contiguous()):
        raise TypeError("expected a contiguous CUDA tensor")
    if str(t.dtype) != "torch." + dtype_name:
        raise TypeError(f"expected torch.{dtype_name}, got {t.dtype}")
    if n is not None and t.numel() != n:
        raise ValueError(f"expected {n} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def _hptr(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(c_vp)


def default_params(**kw):
    p = pgb_params()
    lib().pgb_default_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def pgb_create(params=None, stream=None):
    """stream: a torch.cuda.Stream, a raw cudaStream_t integer or None."""
    h = c_vp()
    s = getattr(stream, "cuda_stream", stream)
    st = lib().pgb_create(ctypes.byref(h), ctypes.byref(params) if params is not None else None,
                          c_vp(s) if s else None)
    _check(None, st)
    return h


def pgb_destroy(ctx):
    return _check(None, lib().pgb_destroy(ctx))


def pgb_last_error(ctx):
    return lib().pgb_last_error(ctx).decode()


def pgb_mesh_load(ctx, kind, verts, tris, eps_in=1.0, charge_xyz=None, charge_q=None, bc_value=0.0):
    v, vp = _hptr(verts, np.float64)
    t, tp = _hptr(tris, np.int32)
    nq = 0 if charge_q is None else len(charge_q)
    if nq:
        qx, qxp = _hptr(charge_xyz, np.float64)
        qq, qqp = _hptr(charge_q, np.float64)
    else:
        qxp = qqp = None
    bid = c_i32()
    _check(ctx, lib().pgb_mesh_load(ctx, kind, vp, v.shape[0], tp, t.shape[0], eps_in, qxp, qqp, nq,
                                    bc_value, ctypes.byref(bid)))
    return bid.value


def pgb_set_solvent(ctx, eps_out, kappa):
    return _check(ctx, lib().pgb_set_solvent(ctx, eps_out, kappa))


def pgb_set_charges(ctx, body_id, q):
    q_, qp = _hptr(np.asarray(q).reshape(-1), np.float64)
    return _check(ctx, lib().pgb_set_charges(ctx, body_id, qp, q_.shape[0]))


def pgb_set_bc(ctx, body_id, bc_value):
    return _check(ctx, lib().pgb_set_bc(ctx, body_id, float(bc_value)))


def pgb_autotune(ctx, thetas, Ps, leaves, reps=5, tol=1e-6, target_rel_err=1e-5):
    """Returns (chosen params dict, report (n, 3): matvec ms, solve ms, energy rel. diff)."""
    th, thp = _hptr(thetas, np.float64)
    pp, ppp = _hptr(Ps, np.int32)
    lv, lvp = _hptr(leaves, np.int32)
    rep = np.zeros((len(th) * len(pp) * len(lv), 3))
    ch = pgb_params()
    _check(ctx, lib().pgb_autotune(ctx, thp, len(th), ppp, len(pp), lvp, len(lv), reps, tol, target_rel_err,
                                   ctypes.byref(ch), rep.ctypes.data_as(c_vp)))
    return {n: getattr(ch, n) for n, _ in pgb_params._fields_}, rep


def pgb_set_region(ctx, body_id, parent, kappa_in=0.0):
    return _check(ctx, lib().pgb_set_region(ctx, body_id, parent, float(kappa_in)))


def pgb_set_pose(ctx, body_id, R, t):
    R_, Rp = _hptr(np.asarray(R).reshape(9), np.float64)
    t_, tp = _hptr(np.asarray(t).reshape(3), np.float64)
    return _check(ctx, lib().pgb_set_pose(ctx, body_id, Rp, tp))


def pgb_tree_build(ctx):
    return _check(ctx, lib().pgb_tree_build(ctx))


def pgb_tree_reset(ctx):
    return _check(ctx, lib().pgb_tree_reset(ctx))


def pgb_tree_refresh(ctx):
    return _check(ctx, lib().pgb_tree_refresh(ctx))


def pgb_tree_stats(ctx):
    info = pgb_tree_info()
    _check(ctx, lib().pgb_tree_stats(ctx, ctypes.byref(info)))
    return {n: getattr(info, n) for n, _ in pgb_tree_info._fields_}


def pgb_num_unknowns(ctx):
    n = c_i64()
    _check(ctx, lib().pgb_num_unknowns(ctx, ctypes.byref(n)))
    return n.value


def pgb_matvec(ctx, x, y, precision):
    n = pgb_num_unknowns(ctx)
    dt = "float32" if precision == PGB_FP32 else "float64"
    return _check(ctx, lib().pgb_matvec(ctx, _dptr(x, dt, n), _dptr(y, dt, n), precision))


def pgb_rhs(ctx, b):
    return _check(ctx, lib().pgb_rhs(ctx, _dptr(b, "float64", pgb_num_unknowns(ctx))))


def pgb_solve(ctx, mode, tol, max_iter, restart, x_out):
    st = pgb_solve_stats()
    code = _check(ctx, lib().pgb_solve(ctx, mode, tol, max_iter, restart,
                                       _dptr(x_out, "float64", pgb_num_unknowns(ctx)), ctypes.byref(st)),
                  allow=(PGB_ENOCONV,))
    return code, {n: getattr(st, n) for n, _ in pgb_solve_stats._fields_}


def pgb_solve_batch(ctx, body_id, R, t, mode, tol, max_iter, restart):
    """R: (B,3,3), t: (B,3) host arrays.  Returns (status, F (B,4) numpy
    [coulomb, solvation, surface, total], list of stats dicts)."""
    R_, Rp = _hptr(np.asarray(R).reshape(-1, 9), np.float64)
    t_, tp = _hptr(np.asarray(t).reshape(-1, 3), np.float64)
    B = R_.shape[0]
    if t_.shape[0] != B:
        raise ValueError("R and t batch sizes differ")
    F = np.zeros((B, 4))
    st = (pgb_solve_stats * max(1, B))()
    code = _check(ctx, lib().pgb_solve_batch(ctx, body_id, Rp, tp, B, mode, tol, max_iter, restart,
                                             F.ctypes.data_as(c_vp), st), allow=(PGB_ENOCONV,))
    return code, F, [{n: getattr(s, n) for n, _ in pgb_solve_stats._fields_} for s in st[:B]]


def pgb_solve_poses(ctxs, pose_ctx, body_id, R, t, mode, tol, max_iter, restart):
    """Poses of several contexts in batches of ctxs[0]'s `batch` parameter:
    pose b is body body_id of ctxs[pose_ctx[b]] at (R[b], t[b]).  Returns
    (status, F (B,4), list of stats dicts) as pgb_solve_batch."""
    R_, Rp = _hptr(np.asarray(R).reshape(-1, 9), np.float64)
    t_, tp = _hptr(np.asarray(t).reshape(-1, 3), np.float64)
    pc_, pcp = _hptr(np.asarray(pose_ctx).reshape(-1), np.int32)
    B = R_.shape[0]
    if t_.shape[0] != B or pc_.shape[0] != B:
        raise ValueError("R, t and pose_ctx batch sizes differ")
    arr = (c_vp * len(ctxs))(*[c.value if isinstance(c, c_vp) else c for c in ctxs])
    F = np.zeros((B, 4))
    st = (pgb_solve_stats * max(1, B))()
    code = _check(ctxs[0], lib().pgb_solve_poses(arr, len(ctxs), pcp, body_id, Rp, tp, B, mode, tol, max_iter,
                                                 restart, F.ctypes.data_as(c_vp), st), allow=(PGB_ENOCONV,))
    return code, F, [{n: getattr(s, n) for n, _ in pgb_solve_stats._fields_} for s in st[:B]]


def pgb_grad(ctx, x, n_charges, n_bodies, precision=PGB_FP32, tol=1e-8, max_iter=1000, restart=100):
    """Adjoint gradients: returns (status, dF_dq (n_charges,), dF_dbc (n_bodies,),
    dF_dt (n_bodies, 3), adjoint stats)."""
    dq = np.zeros(max(1, n_charges))
    dbc = np.zeros(max(1, n_bodies))
    dt = np.zeros((max(1, n_bodies), 3))
    st = pgb_solve_stats()
    code = _check(ctx, lib().pgb_grad(ctx, _dptr(x, "float64", pgb_num_unknowns(ctx)), precision, tol, max_iter,
                                      restart, dq.ctypes.data_as(c_vp), dbc.ctypes.data_as(c_vp),
                                      dt.ctypes.data_as(c_vp), ctypes.byref(st)), allow=(PGB_ENOCONV,))
    return code, dq[:n_charges], dbc[:n_bodies], dt[:n_bodies], {n: getattr(st, n) for n, _ in pgb_solve_stats._fields_}


def pgb_matvec_transpose(ctx, lam, y, precision):
    n = pgb_num_unknowns(ctx)
    return _check(ctx, lib().pgb_matvec_transpose(ctx, _dptr(lam, "float64", n), _dptr(y, "float64", n), precision))


def pgb_energy(ctx, x, n_bodies=None):
    e = pgb_energies()
    per = (pgb_energies * n_bodies)() if n_bodies else None
    _check(ctx, lib().pgb_energy(ctx, _dptr(x, "float64", pgb_num_unknowns(ctx)), ctypes.byref(e), per))
    d = {n: getattr(e, n) for n, _ in pgb_energies._fields_}
    if per is not None:
        d["per_body"] = [{n: getattr(p, n) for n, _ in pgb_energies._fields_} for p in per]
    return d


PGB_NOALLOC_MAX_CHARGES = 65536


def pgb_energy_noalloc(ctx, x):
    """pgb_energy through the entry point that allocates no device memory
    (fixed scratch of PGB_NOALLOC_MAX_CHARGES charges)."""
    e = pgb_energies()
    _check(ctx, lib().pgb_energy_noalloc(ctx, _dptr(x, "float64", pgb_num_unknowns(ctx)), ctypes.byref(e)))
    return {n: getattr(e, n) for n, _ in pgb_energies._fields_}


def pgb_timing(ctx, enable, read=True):
    """Enable/disable stage timing; when read, return and reset the
    accumulated {stage: (ms, calls)}, the kernels run and the host's launch
    calls (direct kernel launches plus graph launches)."""
    t = pgb_stage_times()
    _check(ctx, lib().pgb_timing(ctx, 1 if enable else 0, ctypes.byref(t) if read else None))
    if not read:
        return None
    d = {STAGES[i]: (t.ms[i], t.calls[i]) for i in range(N_STAGES)}
    d["kernel_launches"] = t.kernel_launches
    d["host_launches"] = t.host_launches
    return d


def pgb_tree_export(ctx):
    s = pgb_tree_stats(ctx)
    perm = np.zeros(s["n_panels"], np.int32)
    noff = np.zeros(s["n_groups"] + 1, np.int64)
    foff = np.zeros(s["n_groups"] + 1, np.int64)
    near = np.zeros(max(1, s["n_near"]), np.int32)
    far = np.zeros(max(1, s["n_far"]), np.int32)
    p = lambda a: a.ctypes.data_as(c_vp)
    _check(ctx, lib().pgb_tree_export(ctx, p(perm), p(noff), p(near), p(foff), p(far)))
    return perm, noff, near[:s["n_near"]], foff, far[:s["n_far"]]


def pgb_math_check(x):
    """Device FP64 functions at the points x (host array): columns one-step
    and two-step Newton rsqrt, Taylor exp2, library rsqrt, library exp2,
    double-single rsqrt, double-single exp2."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros((len(x), 7), np.float64)
    _check(None, lib().pgb_math_check(x.ctypes.data_as(c_vp), len(x), out.ctypes.data_as(c_vp)))
    return out


def pgb_alloc_count():
    """Allocations libpgb has made in this process so far (device buffers and
    pinned host buffers); two reads around a call show whether it allocated."""
    n = c_i64()
    _check(None, lib().pgb_alloc_count(ctypes.byref(n)))
    return int(n.value)


def pgb_far_table(P, kappa):
    """(Yukawa, Laplace) far-field tables (T x T each) for order P and kappa."""
    T = (P + 1) * (P + 2) * (P + 3) // 6
    out = np.zeros(2 * T * T)
    _check(None, lib().pgb_far_table(P, float(kappa), out.ctypes.data_as(c_vp), len(out)))
    return out[:T * T].reshape(T, T), out[T * T:].reshape(T, T)


def pgb_orientation_landscape(F, n_orient, n_gap, temperature=300.0):
    """Per separation: dict(most_likely_orientation, p_max, free_energy_kcal_mol)
    from F (n_orient x n_gap energies, orientation-major)."""
    F_, Fp = _hptr(np.asarray(F, dtype=np.float64).reshape(-1), np.float64)
    if F_.shape[0] != n_orient * n_gap:
        raise ValueError("F must hold n_orient * n_gap energies")
    out = np.zeros(3 * n_gap)
    _check(None, lib().pgb_orientation_landscape(Fp, n_orient, n_gap, float(temperature),
                                                 out.ctypes.data_as(c_vp)))
    return [{"gap_index": g, "most_likely_orientation": int(out[3 * g]), "p_max": float(out[3 * g + 1]),
             "free_energy_kcal_mol": float(out[3 * g + 2])} for g in range(n_gap)]


PGB_COLL_ALLGATHER = 0
PGB_COLL_ALLREDUCE = 1


def pgb_shard_partition(work, world):
    """Group bounds (world + 1) of a balanced contiguous split of the work."""
    w, wp = _hptr(np.asarray(work, dtype=np.float64).reshape(-1), np.float64)
    b = np.zeros(world + 1, np.int64)
    _check(None, lib().pgb_shard_partition(wp, w.shape[0], world, b.ctypes.data_as(c_vp)))
    return b


def pgb_shard_rows(ctx, world):
    rb = np.zeros(world + 1, np.int64)
    _check(ctx, lib().pgb_shard_rows(ctx, world, rb.ctypes.data_as(c_vp)))
    return rb


def pgb_to_sharded(ctx, x, xs, inverse=False):
    n = pgb_num_unknowns(ctx)
    return _check(ctx, lib().pgb_to_sharded(ctx, _dptr(x, "float64", n), _dptr(xs, "float64", n), int(inverse)))


def pgb_matvec_shard(ctx, rank, world, xs, ys, precision):
    return _check(ctx, lib().pgb_matvec_shard(ctx, rank, world, _dptr(xs, "float64", pgb_num_unknowns(ctx)),
                                              _dptr(ys, "float64"), precision))


def pgb_solve_shard(ctx, rank, world, xs, red, callback, mode, tol, max_iter, restart, x_out):
    """callback: a ctypes CFUNCTYPE(int, void*, int32, int64) object doing the
    collectives.  Returns (status, stats dict)."""
    n = pgb_num_unknowns(ctx)
    st = pgb_solve_stats()
    code = _check(ctx, lib().pgb_solve_shard(ctx, rank, world, _dptr(xs, "float64", n), _dptr(red, "float64"),
                                             ctypes.cast(callback, c_vp), None, mode, tol, max_iter, restart,
                                             _dptr(x_out, "float64", n), ctypes.byref(st)), allow=(PGB_ENOCONV,))
    return code, {k: getattr(st, k) for k, _ in pgb_solve_stats._fields_}
