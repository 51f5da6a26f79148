"""Context construction from a list of body descriptions (argument
marshalling only): each body is a dict with kind ("dielectric", "sigma" or
"phi"), verts (nv x 3, Angstrom), tris (nt x 3), eps_in, qxyz (nq x 3), q (nq,
e), bc (C/m^2 for "sigma", V for "phi") and optionally a pose R (3 x 3), t (3,)."""
from . import _lib as L

KINDS = {"dielectric": L.PGB_DIELECTRIC, "sigma": L.PGB_SET_CHARGE, "phi": L.PGB_SET_POTENTIAL}


def context(bodies, eps_out=80.0, kappa=0.125, stream=None, build=True, **params):
    """pgb_create + pgb_mesh_load per body (+ pgb_set_pose) + pgb_set_solvent,
    then pgb_tree_build unless build is False.  params override
    pgb_default_params fields; stream is a torch.cuda.Stream, a raw
    cudaStream_t or None (the current torch stream)."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    ctx = L.pgb_create(L.default_params(**params), stream)
    try:
        for b in bodies:
            has_q = len(b["q"]) > 0
            bid = L.pgb_mesh_load(ctx, KINDS[b["kind"]], b["verts"], b["tris"], b["eps_in"],
                                  b["qxyz"] if has_q else None, b["q"] if has_q else None, b["bc"])
            if b.get("R") is not None:
                L.pgb_set_pose(ctx, bid, b["R"], b["t"])
        for bid, b in enumerate(bodies):
            if b.get("parent", -1) != -1 or b.get("kappa_in", 0.0) != 0.0:
                L.pgb_set_region(ctx, bid, b.get("parent", -1), b.get("kappa_in", 0.0))
        L.pgb_set_solvent(ctx, eps_out, kappa)
        if build:
            L.pgb_tree_build(ctx)
    except Exception:
        L.pgb_destroy(ctx)
        raise
    return ctx
