"""Python binding of libmgrit_em.so with the C ABI's names (argument marshalling only).

Device buffers are torch CUDA tensors (float64, contiguous); set-up data are
numpy arrays.  Every computation happens in the library's CUDA kernels.
"""

from __future__ import annotations

import ctypes as C

import numpy as np

from . import lib as L


def _ptr(a) -> C.c_void_p:
    """Address of a contiguous numpy array or torch tensor."""
    if a is None:
        return C.c_void_p(0)
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return C.c_void_p(a.ctypes.data)
    if not a.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return C.c_void_p(a.data_ptr())


def _dev64(t, what: str):
    import torch

    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64):
        raise TypeError(f"{what} must be a CUDA float64 tensor")
    return t


def solver_opts(**kw) -> L.mg_solver_opts:
    lib = L.load()
    so = L.mg_solver_opts()
    lib.mg_solver_defaults(C.byref(so))
    for k, v in kw.items():
        if not hasattr(so, k):
            raise KeyError(k)
        setattr(so, k, v)
    return so


def mgrit_opts(levels=2, m=(16,), space_level=(0, 0), relax=1, tol=1e-10, tol_relative=True, max_iter=50,
               restrict_mode=2, solver: L.mg_solver_opts | None = None, cycle="V", nested=False,
               stop="residual", step_tol_ratio=0.0) -> L.mg_opts:
    lib = L.load()
    o = L.mg_opts()
    lib.mg_opts_defaults(C.byref(o))
    o.levels = levels
    for i, v in enumerate(m):
        o.m[i] = v
    for i, v in enumerate(space_level):
        o.space_level[i] = v
    o.relax = relax
    o.tol = tol
    o.tol_relative = int(bool(tol_relative))
    o.max_iter = max_iter
    o.restrict_mode = restrict_mode
    o.cycle = {"V": 0, "F": 1}[cycle]
    o.nested = 2 if nested == "reference" else int(bool(nested))
    o.stop_rule = {"residual": 0, "joule": 1}[stop]
    o.step_tol_ratio = step_tol_ratio
    if solver is not None:
        o.solver = solver
    return o


def stats_dict(st: L.mg_stats) -> dict:
    return {
        "iters": st.iters,
        "res_hist": [st.res_hist[i] for i in range(st.n_hist)],
        "t_setup": st.t_setup,
        "t_solve": st.t_solve,
        "step_solves": st.step_solves,
        "batched_steps": st.batched_steps,
        "cg_iters": st.cg_iters,
        "worst_status": L.STATUS.get(st.worst_status, st.worst_status),
        "launches": st.launches,
        "newton_iters": st.newton_iters,
    }


class Context:
    """One mg_ctx on a CUDA device, bound to a CUDA stream (torch's current by default)."""

    def __init__(self, device: int = 0, stream=None):
        import torch

        self.lib = L.load()
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = C.c_void_p()
        self.h = None
        self._check(self.lib.mg_create(C.byref(h), device, C.c_void_p(stream.cuda_stream)))
        self.h = h

    # -------------------------------------------------------------- helpers
    def _check(self, st: int, allow=()) -> int:
        if st != L.MG_OK and st not in allow:
            msg = self.lib.mg_last_error(self.h) if self.h else b"mg_create failed"
            raise L.MgError(st, (msg or b"").decode())
        return st

    def close(self):
        if getattr(self, "h", None):
            self.lib.mg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -------------------------------------------------------------- set-up
    def mg_add_mesh(self, xy, tri, region, dirichlet) -> int:
        xy = np.ascontiguousarray(xy, dtype=np.float64)
        tri = np.ascontiguousarray(tri, dtype=np.int32)
        region = np.ascontiguousarray(region, dtype=np.int32)
        dirichlet = np.ascontiguousarray(dirichlet, dtype=np.int32)
        lvl = C.c_int()
        self._check(self.lib.mg_add_mesh(self.h, C.byref(lvl), xy.shape[0], _ptr(xy), tri.shape[0], _ptr(tri),
                                         _ptr(region), dirichlet.size, _ptr(dirichlet)))
        return lvl.value

    def mg_add_refinement(self, fine: int, coarse: int, parent):
        parent = np.ascontiguousarray(parent, dtype=np.int32)
        self._check(self.lib.mg_add_refinement(self.h, fine, coarse, _ptr(parent)))

    def mg_add_transfer(self, fine: int, coarse: int, rowptr, col, val):
        """P_s (fine <- coarse) as node-indexed CSR arrays (e.g. a scipy csr_matrix's
        indptr, indices, data)."""
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
        val = np.ascontiguousarray(val, dtype=np.float64)
        self._check(self.lib.mg_add_transfer(self.h, fine, coarse, int(rowptr[-1]), _ptr(rowptr), _ptr(col),
                                             _ptr(val)))

    def mg_set_material(self, region, sigma, nu, law=0, k1=0.0, k2=0.0, k3=0.0):
        self._check(self.lib.mg_set_material(self.h, region, sigma, nu, law, k1, k2, k3))

    def mg_set_source(self, region, phase, sign):
        self._check(self.lib.mg_set_source(self.h, region, phase, sign))

    def mg_set_pwm(self, J0, f_ref, f_carrier, carrier, mod_index):
        self._check(self.lib.mg_set_pwm(self.h, J0, f_ref, f_carrier, carrier, mod_index))

    def mg_plan_levels(self, fine_level, coarse_level, N, T, max_levels=5, opts=None):
        """Returns (mg_opts with levels, m, space_level filled, estimated ms per FCF iteration)."""
        o = opts or mgrit_opts()
        ms = C.c_double(0.0)
        self._check(self.lib.mg_plan_levels(self.h, fine_level, coarse_level, N, T, max_levels, C.byref(o),
                                            C.byref(ms)))
        return o, ms.value

    def mg_set_ramp(self, t_ramp):
        self._check(self.lib.mg_set_ramp(self.h, t_ramp))

    def mg_joule_losses(self, level, N, T, traj, losses):
        _dev64(traj, "traj")
        _dev64(losses, "losses")
        self._check(self.lib.mg_joule_losses(self.h, level, N, T, _ptr(traj), _ptr(losses)))

    def mg_finalize(self):
        self._check(self.lib.mg_finalize(self.h))

    def mg_num_dofs(self, level: int) -> int:
        return int(self.lib.mg_num_dofs(self.h, level))

    def mg_get_operators(self, level: int) -> dict:
        n = self.mg_num_dofs(level)
        nnz = C.c_int64()
        self._check(self.lib.mg_get_operators(self.h, level, C.byref(nnz), None, None, None, None, None))
        rowptr = np.empty(n + 1, np.int64)
        col = np.empty(nnz.value, np.int32)
        K = np.empty(nnz.value)
        M = np.empty(nnz.value)
        F = np.empty(3 * n)
        self._check(self.lib.mg_get_operators(self.h, level, C.byref(nnz), _ptr(rowptr), _ptr(col), _ptr(K),
                                              _ptr(M), _ptr(F)))
        return {"rowptr": rowptr, "col": col, "K": K, "M": M, "F": F.reshape(3, n)}

    def mg_pwm_table(self, N: int, T: float) -> np.ndarray:
        out = np.empty((N + 1, 3), np.int8)
        self._check(self.lib.mg_pwm_table(self.h, N, T, _ptr(out)))
        return out

    # -------------------------------------------------------------- solving
    def mg_step(self, level, N, T, x_in, x_out, dt_mult=1, i0=1, istride=0, guess=False, solver=None,
                allow=()):
        _dev64(x_in, "x_in")
        _dev64(x_out, "x_out")
        k = x_out.shape[1] if x_out.dim() == 2 else 1
        ld_in = x_in.shape[1] if x_in.dim() == 2 else 1
        ld_out = k
        st = L.mg_stats()
        so = solver or solver_opts()
        rc = self.lib.mg_step(self.h, level, N, T, dt_mult, k, i0, istride, _ptr(x_in), ld_in, _ptr(x_out), ld_out,
                              int(bool(guess)), C.byref(so), C.byref(st))
        self._check(rc, allow=allow)
        return rc, stats_dict(st)

    def mg_step_static(self, level, N, T, x_in, x_out, dt_mult=1, i0=1, istride=0, guess=False, solver=None,
                       allow=()):
        _dev64(x_in, "x_in")
        _dev64(x_out, "x_out")
        k = x_out.shape[1] if x_out.dim() == 2 else 1
        ld_in = x_in.shape[1] if x_in.dim() == 2 else 1
        st = L.mg_stats()
        so = solver or solver_opts()
        rc = self.lib.mg_step_static(self.h, level, N, T, dt_mult, k, i0, istride, _ptr(x_in), ld_in, _ptr(x_out),
                                     k, int(bool(guess)), C.byref(so), C.byref(st))
        self._check(rc, allow=allow)
        return rc, stats_dict(st)

    def mg_autotune(self, level, N, T, k, solver=None):
        """Returns (tuned solver options, ms per step of the chosen launch shape)."""
        so = solver or solver_opts()
        ms = C.c_double(0.0)
        rc = self.lib.mg_autotune(self.h, level, N, T, k, C.byref(so), C.byref(ms))
        self._check(rc)
        return so, ms.value

    def mg_sequential(self, level, N, T, a0, out, solver=None, allow=()):
        _dev64(a0, "a0")
        _dev64(out, "out")
        st = L.mg_stats()
        so = solver or solver_opts()
        rc = self.lib.mg_sequential(self.h, level, N, T, _ptr(a0), _ptr(out), C.byref(so), C.byref(st))
        self._check(rc, allow=allow)
        return rc, stats_dict(st)

    def mg_solve(self, N, T, a0, out, opts: L.mg_opts, allow=(), stats=True):
        _dev64(a0, "a0")
        _dev64(out, "out")
        st = L.mg_stats()
        rc = self.lib.mg_solve(self.h, N, T, _ptr(a0), _ptr(out), C.byref(opts),
                               C.byref(st) if stats else None)
        self._check(rc, allow=allow)
        return rc, stats_dict(st)

    def mg_solve_work_bytes(self, N, opts: L.mg_opts) -> int:
        """Estimated device bytes of the work buffers mg_solve allocates for N steps."""
        b = C.c_int64(0)
        self._check(self.lib.mg_solve_work_bytes(self.h, N, C.byref(opts), C.byref(b)))
        return b.value

    def mg_release_work(self):
        """Free the context's work buffers (step plans, solve storage); meshes and operators stay."""
        self._check(self.lib.mg_release_work(self.h))

    def mg_solve_host(self, N, T, a0: np.ndarray, out: np.ndarray, opts: L.mg_opts, allow=()):
        assert a0.dtype == np.float64 and out.dtype == np.float64
        st = L.mg_stats()
        rc = self.lib.mg_solve_host(self.h, N, T, _ptr(a0), _ptr(out), C.byref(opts), C.byref(st))
        self._check(rc, allow=allow)
        return rc, stats_dict(st)

    def mg_sequential_host(self, level, N, T, a0: np.ndarray, out: np.ndarray, solver=None, allow=()):
        st = L.mg_stats()
        so = solver or solver_opts()
        rc = self.lib.mg_sequential_host(self.h, level, N, T, _ptr(a0), _ptr(out), C.byref(so), C.byref(st))
        self._check(rc, allow=allow)
        return rc, stats_dict(st)


def setup_machine(ctx: Context, meshes, model) -> list:
    """Hand a synthetic machine (synth.mesh_hierarchy + synth.machine_model) to the library.

    Returns the library's level id of each mesh.  Pure data marshalling.
    """
    ids = []
    for m in meshes:
        ids.append(ctx.mg_add_mesh(m.xy, m.tri, m.region, m.dirichlet_nodes()))
    for k in range(1, len(meshes)):
        ctx.mg_add_refinement(ids[k], ids[k - 1], meshes[k].parent)
    for r, mat in enumerate(model.materials):
        ctx.mg_set_material(r, mat.sigma, mat.nu, mat.law, mat.k1, mat.k2, mat.k3)
    for region, phase, sign in model.coil_phase:
        ctx.mg_set_source(region, phase, sign)
    p = model.pwm
    ctx.mg_set_pwm(p.J0, p.f_ref, p.f_carrier, p.carrier, p.mod_index)
    return ids


def mg_batch_solve(ctxs, N, T, a0, out, opts, max_threads=0, work_budget=0):
    """Solve independent instances concurrently (one Context each, distinct streams).

    N, T, a0, out, opts: one entry per instance (a0/out device tensors as for
    Context.mg_solve).  work_budget: device bytes the running instances' work
    buffers may take together (0: no limit, -1: the free device memory; see
    mg_batch_solve in the header).  Returns (worst status, [status], [stats dict]).
    """
    n = len(ctxs)
    lib = L.load()
    for a, o in zip(a0, out):
        _dev64(a, "a0")
        _dev64(o, "out")
    hs = (C.c_void_p * n)(*[c.h.value if isinstance(c.h, C.c_void_p) else c.h for c in ctxs])
    Ns = (C.c_int64 * n)(*N)
    Ts = (C.c_double * n)(*T)
    a0p = (C.c_void_p * n)(*[a.data_ptr() for a in a0])
    outp = (C.c_void_p * n)(*[o.data_ptr() for o in out])
    op = (L.mg_opts * n)(*opts)
    st = (C.c_int * n)()
    stats = (L.mg_stats * n)()
    rc = lib.mg_batch_solve(hs, n, Ns, Ts, a0p, outp, op, max_threads, work_budget, st, stats)
    return rc, [L.STATUS.get(v, v) for v in st], [stats_dict(s) for s in stats]


def mg_smoother_weights(lam, nu, solver=None):
    """Weights of one pre-smoothing of nu sweeps on a depth with Gershgorin bound
    lam (host only): Chebyshev roots on [lam / cheb_ratio, lam] or omega."""
    lib = L.load()
    so = solver or solver_opts()
    w = (C.c_float * max(1, nu))()
    rc = lib.mg_smoother_weights(C.byref(so), lam, nu, w)
    if rc != L.MG_OK:
        raise L.MgError(rc, "mg_smoother_weights: bad input")
    return [w[i] for i in range(nu)]


def mg_choose_levels(k_list, ms_list, N, max_levels=5, coarse_m=0):
    """Sec. 4.1's coarsening heuristic on measured step times (host only); coarse_m
    is the factor below the first level (0: 2).  Returns (levels, [m_0, ..., m_{levels-2}])."""
    lib = L.load()
    nk = len(k_list)
    ks = (C.c_double * nk)(*k_list)
    ts = (C.c_double * nk)(*ms_list)
    lv = C.c_int(0)
    m = (C.c_int * 8)()
    rc = lib.mg_choose_levels(ks, ts, nk, N, max_levels, coarse_m, C.byref(lv), m)
    if rc != L.MG_OK:
        raise L.MgError(rc, "mg_choose_levels: bad input")
    return lv.value, [m[i] for i in range(lv.value - 1)]
