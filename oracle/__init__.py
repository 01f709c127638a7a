"""ORACLE -- test infrastructure only.

A plain, slow FP64 CPU restatement of the electrostatic PIC-MCC particle cycle on a
cell-based quadtree of Kolobov & Arslanbekov, "Electrostatic PIC with adaptive Cartesian
mesh" (arXiv:1604.07713).  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import it.  It shares no code with the
CUDA path and imports nothing from the package.

Per-particle and per-leaf loops live in ``pic_oracle.c`` (plain C, FP64, no FMA
contraction); this module holds the step order, the cell-list bookkeeping and the
Poisson solve (scipy sparse direct solve of the assembled operator).

Step order for step n (one reading of §3 / §3.1, applied identically by the CUDA path):
  deposit (NGP, §3) -> Poisson (§3) -> node E (§3) -> push + walls + location + MCC
  (§3, §3.1) -> cell-list update (§3.1: a particle that leaves a cell is removed from its
  list and appended to the list of the cell it enters; spawned pairs are appended after).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "pic_oracle.c"), os.path.join(_HERE, "pic_oracle_adapt.c")]
_LIB_PATH = os.path.join(_HERE, "_liboracle.so")

BC_PERIODIC, BC_DIRICHLET, BC_NEUMANN = 0, 1, 2
QE = 1.602176634e-19
ME = 9.1093837015e-31
AMU = 1.66053906660e-27
EPS0 = 8.8541878128e-12


def build(force: bool = False) -> str:
    """Compile the oracle's C core with gcc (FP64, no fused multiply-add)."""
    srcs = [s for s in _SRC if os.path.exists(s)]
    newest = max(os.path.getmtime(s) for s in srcs)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", *srcs, "-lm", "-o", tmp]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


_p = C.c_void_p
_i64 = C.c_int64
_i32 = C.c_int32
_u32 = C.c_uint32


class _Mesh(C.Structure):
    _fields_ = [("nx0", _i32), ("ny0", _i32), ("lmax", _i32), ("bc_x", _i32), ("bc_y", _i32),
                ("pad_", _i32), ("h0", C.c_double), ("nleaf", _i64), ("key", _p), ("ix", _p),
                ("iy", _p), ("s", _p)]


class _PushParams(C.Structure):
    _fields_ = [("dt", C.c_double), ("q", C.c_double), ("m", C.c_double), ("species", _i32),
                ("mcc", _i32), ("ng", C.c_double), ("sigma_el", C.c_double),
                ("sigma_iz0", C.c_double), ("eps_th_ev", C.c_double), ("qe", C.c_double),
                ("m_neutral", C.c_double), ("t_gas_ev", C.c_double), ("key0", _u32),
                ("key1", _u32), ("inst", _u32), ("step", _u32), ("lx", C.c_double),
                ("ly", C.c_double), ("mode", _i32)]


def _declare(L):
    L.or_philox4x32_10.argtypes = [_p, _p, _p]
    L.or_philox2x32_10.argtypes = [_p, _u32, _p]
    L.or_philox_bulk.argtypes = [_i64, _p, _u32, _u32, _u32, _u32, _u32, _p]
    L.or_morton.argtypes = [_u32, _u32]
    L.or_morton.restype = _u32
    L.or_leaf_geometry.argtypes = [_i64, _i32, _i32, _i32, _p, _p, _p, _p, _p, _p, _p]
    L.or_leaf_geometry.restype = C.c_int
    L.or_locate.argtypes = [C.POINTER(_Mesh), _i64, _p, _p, _p]
    L.or_locate_brute.argtypes = [C.POINTER(_Mesh), _i64, _p, _p, _p]
    L.or_leaf_at.argtypes = [C.POINTER(_Mesh), _i32, _i32]
    L.or_leaf_at.restype = _i64
    L.or_check_tree.argtypes = [C.POINTER(_Mesh)]
    L.or_check_tree.restype = C.c_int
    L.or_face_table.argtypes = [C.POINTER(_Mesh), _p, _p, _p, _p]
    L.or_assemble.argtypes = [C.POINTER(_Mesh), _p, _p, _p, _p]
    L.or_assemble.restype = _i64
    L.or_node_e.argtypes = [C.POINTER(_Mesh), _p, _p, _p]
    L.or_cell_emag.argtypes = [C.POINTER(_Mesh), _p, _p, _p]
    L.or_deposit.argtypes = [_i64, _i64, _p, _p, C.c_double, _p]
    L.or_push_mcc.argtypes = [C.POINTER(_Mesh), C.POINTER(_PushParams), _p, _i64, _p, _p, _p,
                              _p, _p, _p, _p, _p, _p, _p, _p, _p, _p]
    L.or_cic_deposit.argtypes = [_i32, _i32, C.c_double, _i32, _i32, _i64, _p, _p, _p, C.c_double, _p]
    L.or_cic_gather.argtypes = [_i32, _i32, C.c_double, _i32, _i32, _p, _p, _i32, _i64, _p, _p, _p, _p]
    L.or_push_mcc.restype = _i64
    L.or_assemble_kappa.argtypes = [C.POINTER(_Mesh), _p, _p, _p, _p, _p]
    L.or_assemble_kappa.restype = _i64


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def philox2(ctr0: int, ctr1: int, key: int):
    """Philox2x32-10 of one counter (Salmon et al., SC'11): the two output words."""
    c = np.array([ctr0, ctr1], np.uint32)
    out = np.zeros(2, np.uint32)
    lib().or_philox2x32_10(_ptr(c), key & 0xFFFFFFFF, _ptr(out))
    return int(out[0]), int(out[1])


# ---------------------------------------------------------------------------------------
# Philox4x32-10 (Salmon et al., SC'11)
# ---------------------------------------------------------------------------------------
def philox(ctr0: np.ndarray, ctr1: int, ctr2: int, ctr3: int, key0: int, key1: int) -> np.ndarray:
    c0 = np.ascontiguousarray(ctr0, dtype=np.uint32)
    out = np.empty((c0.size, 4), np.uint32)
    lib().or_philox_bulk(c0.size, _ptr(c0), ctr1, ctr2, ctr3, key0, key1, _ptr(out))
    return out


def uniform24(r: np.ndarray) -> np.ndarray:
    """Top 24 bits scaled to [0, 1): exact in FP32 and FP64."""
    return (r >> 8).astype(np.float64) * (1.0 / 16777216.0)


def morton(cx: int, cy: int) -> int:
    return int(lib().or_morton(cx, cy))


# ---------------------------------------------------------------------------------------
# Quadtree leaf mesh (forest of nx0 x ny0 roots, §2.1 FOT + Morton SFC; §3.1 quad-tree)
# ---------------------------------------------------------------------------------------
class Mesh:
    """Leaves of a forest of quadtrees, stored in ascending Morton key order."""

    def __init__(self, nx0, ny0, h0, lmax, bc_x, bc_y, root=None, level=None, morton_code=None,
                 check=True):
        self.nx0, self.ny0, self.h0, self.lmax = int(nx0), int(ny0), float(h0), int(lmax)
        self.bc_x, self.bc_y = int(bc_x), int(bc_y)
        if root is None:
            n = self.nx0 * self.ny0
            root = np.arange(n, dtype=np.int32)
            level = np.zeros(n, np.int32)
            morton_code = np.zeros(n, np.uint32)
        root = np.ascontiguousarray(root, np.int32)
        level = np.ascontiguousarray(level, np.int32)
        morton_code = np.ascontiguousarray(morton_code, np.uint32)
        n = root.size
        ix = np.empty(n, np.int32); iy = np.empty(n, np.int32); s = np.empty(n, np.int32)
        key = np.empty(n, np.int64)
        rc = lib().or_leaf_geometry(n, self.nx0, self.ny0, self.lmax, _ptr(root), _ptr(level),
                                    _ptr(morton_code), _ptr(ix), _ptr(iy), _ptr(s), _ptr(key))
        if rc != 0:
            raise ValueError("invalid leaf description")
        order = np.argsort(key, kind="stable")
        self.root, self.level, self.morton = root[order], level[order], morton_code[order]
        self.ix, self.iy, self.s, self.key = ix[order], iy[order], s[order], key[order]
        self.nleaf = n
        self._c = _Mesh(self.nx0, self.ny0, self.lmax, self.bc_x, self.bc_y, 0, self.h0, n,
                        _ptr(self.key), _ptr(self.ix), _ptr(self.iy), _ptr(self.s))
        if check:
            rc = lib().or_check_tree(C.byref(self._c))
            if rc != 0:
                raise ValueError(f"leaf set is not a 2:1-balanced tiling (code {rc})")

    @property
    def hf(self):
        return self.h0 / (1 << self.lmax)

    @property
    def lx(self):
        return self.nx0 * self.h0

    @property
    def ly(self):
        return self.ny0 * self.h0

    def h(self):
        return self.s * self.hf

    def area(self):
        return (self.s * self.hf) ** 2

    def centres(self):
        h = self.s * self.hf
        return self.ix * self.hf + 0.5 * h, self.iy * self.hf + 0.5 * h

    def locate(self, x, y, brute=False):
        x = np.ascontiguousarray(x, np.float64); y = np.ascontiguousarray(y, np.float64)
        out = np.empty(x.size, np.int64)
        f = lib().or_locate_brute if brute else lib().or_locate
        f(C.byref(self._c), x.size, _ptr(x), _ptr(y), _ptr(out))
        return out

    def leaf_at(self, I, J):
        return int(lib().or_leaf_at(C.byref(self._c), int(I), int(J)))

    def face_table(self):
        n = self.nleaf
        t = np.empty(4 * n, np.int32); a = np.empty(4 * n, np.int64)
        b = np.empty(4 * n, np.int64); sb = np.empty(4 * n, np.int64)
        lib().or_face_table(C.byref(self._c), _ptr(t), _ptr(a), _ptr(b), _ptr(sb))
        return t.reshape(n, 4), a.reshape(n, 4), b.reshape(n, 4), sb.reshape(n, 4)

    # -- Poisson operator (§3) -------------------------------------------------------
    def operator(self):
        """Composite-mesh operator A (sum of face conductances, divided by eps0) and the
        Dirichlet wall coefficients bc[l, wall]: A phi = rho h^2/eps0 + sum bc * phi_wall."""
        if getattr(self, "_op", None) is None:
            import scipy.sparse as sp
            n = self.nleaf
            cap = 9 * n
            row = np.empty(cap, np.int64); col = np.empty(cap, np.int64)
            val = np.empty(cap, np.float64); bc = np.empty(4 * n, np.float64)
            k = lib().or_assemble(C.byref(self._c), _ptr(row), _ptr(col), _ptr(val), _ptr(bc))
            if k < 0:
                raise ValueError("unbalanced tree")
            A = sp.csr_matrix((val[:k], (row[:k], col[:k])), shape=(n, n))
            A.sum_duplicates()
            self._op = (A, bc.reshape(n, 4))
        return self._op

    def operator_kappa(self, kappa):
        """The operator with a relative permittivity ``kappa`` per leaf (the direct implicit
        scheme's 1 + chi, §3): each face's conductance times the face's kappa (or_assemble_kappa)."""
        import scipy.sparse as sp
        n = self.nleaf
        cap = 9 * n
        kap = np.ascontiguousarray(kappa, np.float64)
        row = np.empty(cap, np.int64); col = np.empty(cap, np.int64)
        val = np.empty(cap, np.float64); bc = np.empty(4 * n, np.float64)
        k = lib().or_assemble_kappa(C.byref(self._c), _ptr(kap), _ptr(row), _ptr(col), _ptr(val), _ptr(bc))
        if k < 0:
            raise ValueError("unbalanced tree")
        A = sp.csr_matrix((val[:k], (row[:k], col[:k])), shape=(n, n))
        A.sum_duplicates()
        return A, bc.reshape(n, 4)

    def solve_poisson(self, rhs_charge_over_eps0, walls, kappa=None):
        """Solve A phi = b on the leaves (sparse direct, FP64).  ``rhs_charge_over_eps0`` is
        rho*h^2/eps0 per leaf, ``walls`` = (phi_x_lo, phi_x_hi, phi_y_lo, phi_y_hi).
        A fully periodic mesh is solved for the zero-mean potential (bordered system).  With
        ``kappa`` the operator is the relative-permittivity one (operator_kappa)."""
        import scipy.sparse as sp
        import scipy.sparse.linalg as spla
        A, bc = self.operator() if kappa is None else self.operator_kappa(kappa)
        b = np.asarray(rhs_charge_over_eps0, np.float64) + bc @ np.asarray(walls, np.float64)
        if self.bc_x == BC_PERIODIC and self.bc_y == BC_PERIODIC:
            n = self.nleaf
            area = self.area() / self.area().sum()
            B = sp.bmat([[A, sp.csr_matrix(area.reshape(n, 1))],
                         [sp.csr_matrix(area.reshape(1, n)), None]], format="csc")
            sol = spla.spsolve(B, np.concatenate([b, [0.0]]))
            return np.asarray(sol[:n])
        return np.asarray(spla.spsolve(A.tocsc(), b))

    def node_e(self, phi, walls):
        phi = np.ascontiguousarray(phi, np.float64)
        w = np.ascontiguousarray(walls, np.float64)
        out = np.empty(8 * self.nleaf, np.float64)
        lib().or_node_e(C.byref(self._c), _ptr(phi), _ptr(w), _ptr(out))
        return out.reshape(self.nleaf, 4, 2)

    def cell_emag(self, phi, walls):
        phi = np.ascontiguousarray(phi, np.float64)
        w = np.ascontiguousarray(walls, np.float64)
        out = np.empty(self.nleaf, np.float64)
        lib().or_cell_emag(C.byref(self._c), _ptr(phi), _ptr(w), _ptr(out))
        return out


def uniform_mesh(nx0, ny0, h0, bc_x, bc_y, lmax=0):
    return Mesh(nx0, ny0, h0, lmax, bc_x, bc_y)


# ---------------------------------------------------------------------------------------
# Particles and the step
# ---------------------------------------------------------------------------------------
class Species:
    """One species' cell lists: arrays kept in list order (leaf ascending; inside a leaf,
    the order of arrival)."""

    def __init__(self, q, m, x, y, vx, vy, vz, w, ids, leaf):
        self.q, self.m = float(q), float(m)
        self.x, self.y = x, y
        self.vx, self.vy, self.vz, self.w, self.id, self.leaf = vx, vy, vz, w, ids, leaf

    @property
    def n(self):
        return self.x.size

    def take(self, idx):
        return Species(self.q, self.m, self.x[idx], self.y[idx], self.vx[idx], self.vy[idx],
                       self.vz[idx], self.w[idx], self.id[idx], self.leaf[idx])


def philox_key(seed: int):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32


class Sim:
    """FP64 oracle of one PIC-MCC instance.

    ``cfg`` is a plain dict with the keys of the C-ABI's configuration (SI or normalised
    units): dt, eps0, q (list), m (list), mcc, gas_density, gas_temperature_ev,
    neutral_mass, sigma_el, sigma_iz0, eps_th_ev, qe, bc_x, bc_y, phi_left_dc,
    phi_left_amp, phi_left_freq, phi_right, rho_background, seed, instance.
    """

    def __init__(self, cfg: dict, mesh: Mesh):
        self.cfg = dict(cfg)
        self.mesh = mesh
        self.step_count = 0
        self.next_id = 0
        self.species: list[Species | None] = [None] * len(self.cfg["q"])
        self.phi = np.zeros(mesh.nleaf)
        self.last_walls = None
        self.last_rho = None
        self.last_node_e = None
        self.last_decisions = {}
        self.diag = None

    # -- loading: the population is located and put into list order by a stable sort on
    #    the leaf index (load order inside a leaf) ---------------------------------------
    def load(self, s, x, y, vx, vy, vz, w, ids=None):
        x = np.array(x, np.float64); y = np.array(y, np.float64)
        n = x.size
        if ids is None:
            ids = np.arange(self.next_id, self.next_id + n, dtype=np.uint64)
        ids = np.array(ids, np.uint64)
        if n:
            self.next_id = max(self.next_id, int(ids.max()) + 1)
        leaf = self.mesh.locate(x, y)
        if np.any(leaf < 0):
            raise ValueError("particle outside the domain")
        order = np.argsort(leaf, kind="stable")
        sp = Species(self.cfg["q"][s], self.cfg["m"][s], x, y, np.array(vx, np.float64),
                     np.array(vy, np.float64), np.array(vz, np.float64), np.array(w, np.float64),
                     ids, leaf)
        self.species[s] = sp.take(order)

    def walls(self, step=None):
        c = self.cfg
        n = self.step_count if step is None else step
        t = n * c["dt"]
        lo = c.get("phi_left_dc", 0.0) + c.get("phi_left_amp", 0.0) * np.sin(
            2.0 * np.pi * c.get("phi_left_freq", 0.0) * t)
        return np.array([lo, c.get("phi_right", 0.0), 0.0, 0.0])

    # -- §3 NGP deposit -------------------------------------------------------------------
    def shape(self):
        """0: NGP deposit with the bilinear corner gather; 1: CIC-EM; 2: CIC-EC (§3, uniform
        meshes only)."""
        sh = int(self.cfg.get("shape", 0))
        if sh and self.mesh.lmax != 0:
            raise ValueError("cloud-in-cell shapes need a uniform mesh")
        return sh

    def charge(self):
        Q = np.zeros(self.mesh.nleaf)
        M = self.mesh
        for sp in self.species:
            if sp is None or sp.n == 0:
                continue
            if self.shape():
                # uniform mesh: leaf index = i + j nx0 (Morton order of the roots is row-major)
                lib().or_cic_deposit(M.nx0, M.ny0, M.h0, int(M.bc_x == BC_PERIODIC),
                                     int(M.bc_y == BC_PERIODIC), sp.n, _ptr(sp.x), _ptr(sp.y),
                                     _ptr(sp.w), sp.q, _ptr(Q))
            else:
                lib().or_deposit(self.mesh.nleaf, sp.n, _ptr(sp.leaf), _ptr(sp.w), sp.q, _ptr(Q))
        return Q

    def cic_field(self, sp, phi=None, walls=None):
        """(ex, ey) at the particles of ``sp`` with the cloud-in-cell shape of the config."""
        M = self.mesh
        phi = np.ascontiguousarray(self.phi if phi is None else phi, np.float64)
        w = np.ascontiguousarray(self.last_walls if walls is None else walls, np.float64)
        ex = np.empty(sp.n); ey = np.empty(sp.n)
        lib().or_cic_gather(M.nx0, M.ny0, M.h0, M.bc_x, M.bc_y, _ptr(phi), _ptr(w), self.shape(), sp.n,
                            _ptr(sp.x), _ptr(sp.y), _ptr(ex), _ptr(ey))
        return ex, ey

    def rho(self):
        return self.charge() / self.mesh.area() + self.cfg.get("rho_background", 0.0)

    # -- §3 direct implicit PIC (DIPIC) ---------------------------------------------------
    def implicit(self):
        """True when the config selects the direct implicit scheme (NGP only)."""
        on = bool(self.cfg.get("implicit", 0))
        if on and self.shape():
            raise ValueError("the implicit scheme uses the NGP shape")
        return on

    def kappa(self):
        """The implicit susceptibility as a relative permittivity per leaf: 1 + chi with
        chi = dt^2 sum_s q_s^2 n_s / (m_s eps0) = (omega_ps dt)^2 summed over species, n_s the
        species' weight per area in the leaf (at the predicted positions during a step)."""
        c = self.cfg
        M = self.mesh
        chi = np.zeros(M.nleaf)
        for sp in self.species:
            if sp is None or sp.n == 0:
                continue
            W = np.bincount(sp.leaf, weights=sp.w, minlength=M.nleaf)
            chi += (c["dt"] ** 2 * sp.q ** 2 / (sp.m * c["eps0"])) * W
        return 1.0 + chi / M.area()

    def fields(self):
        """Deposit -> Poisson -> node E for the current state (no particle update).  With the
        implicit scheme the Poisson operator carries the susceptibility of the current state."""
        rho = self.rho()
        b = rho * self.mesh.area() / self.cfg["eps0"]
        walls = self.walls()
        phi = self.mesh.solve_poisson(b, walls, self.kappa() if self.implicit() else None)
        E = self.mesh.node_e(phi, walls)
        self.phi, self.last_rho, self.last_node_e, self.last_walls = phi, rho, E, walls
        return rho, phi, E

    # -- §3.1 / §4.3 adaptation and particle management (oracle/adapt.py) ----------------
    def adapt(self, mesh=True, particles=True):
        from .adapt import adapt_mesh, split_merge
        out = {}
        if mesh:
            out["mesh"] = adapt_mesh(self)
            if out["mesh"]["refined"] or out["mesh"]["coarsened"]:
                self.diag_reset()  # §3.1: statistics counters restart when the grid changes
        if particles:
            out["particles"] = split_merge(self)
        return out

    # -- §3.3 time averages: the discharge's RF-cycle averages of n_e, n_i, T_e, phi and the
    #    electron energy distribution, accumulated over the steps since the last reset ----
    def diag_enable(self, n_bins, eps_max_ev, region=None):
        """Every later step samples, after its field solve, the stored state (x^n,
        v^{n-1/2}) and the step's potential: per leaf the electron and ion weights, the
        electrons' weighted kinetic energy eps = m |v|^2 / (2 qe) [eV] and phi; and the weight
        of every electron inside region (x0, x1, y0, y1; [x0, x1) x [y0, y1)) goes to the
        energy bin floor(eps * (n_bins / eps_max)) when that is below n_bins."""
        if n_bins <= 0:
            self.diag = None
            return
        r = (-np.inf, np.inf, -np.inf, np.inf) if region is None else tuple(float(v) for v in region)
        self.diag = dict(n_bins=int(n_bins), eps_max=float(eps_max_ev), region=r)
        self.diag_reset()

    def diag_reset(self):
        d = self.diag
        if d is None:
            return
        n = self.mesh.nleaf
        d.update(we=np.zeros(n), wi=np.zeros(n), wee=np.zeros(n), phi=np.zeros(n),
                 hist=np.zeros(d["n_bins"]), samples=0)

    def _diag_sample(self):
        d = self.diag
        e = self.species[0]
        if e is not None and e.n:
            hmq = 0.5 * e.m / self.cfg.get("qe", QE)
            eps = hmq * (e.vx * e.vx + e.vy * e.vy + e.vz * e.vz)
            np.add.at(d["we"], e.leaf, e.w)
            np.add.at(d["wee"], e.leaf, e.w * eps)
            x0, x1, y0, y1 = d["region"]
            inside = (e.x >= x0) & (e.x < x1) & (e.y >= y0) & (e.y < y1) & (eps < d["eps_max"])
            b = np.floor(eps[inside] * (d["n_bins"] / d["eps_max"])).astype(np.int64)
            keep = b < d["n_bins"]
            np.add.at(d["hist"], b[keep], e.w[inside][keep])
        if len(self.species) > 1 and self.species[1] is not None and self.species[1].n:
            np.add.at(d["wi"], self.species[1].leaf, self.species[1].w)
        d["phi"] += self.phi
        d["samples"] += 1

    def diag_fields(self):
        """Averages since the reset: n_e, n_i [per volume], T_e = (2/3) <eps> [eV], phi."""
        d = self.diag
        k = max(1, d["samples"])
        area = self.mesh.area()
        z = d["samples"] > 0
        te = np.where(d["we"] > 0, (2.0 / 3.0) * d["wee"] / np.where(d["we"] > 0, d["we"], 1.0), 0.0)
        return dict(ne=d["we"] / (k * area) * z, ni=d["wi"] / (k * area) * z, te=te * z, phi=d["phi"] / k * z)

    def diag_eedf(self):
        """f[b] = S_b / (sum S * d_eps) [1/eV] and the number of samples."""
        d = self.diag
        tot = d["hist"].sum()
        deps = d["eps_max"] / d["n_bins"]
        f = d["hist"] / (tot * deps) if tot > 0 else np.zeros(d["n_bins"])
        return f, d["samples"]

    def push_params(self, s, mode=0):
        c = self.cfg
        k0, k1 = philox_key(c.get("seed", 0))
        return _PushParams(c["dt"], c["q"][s], c["m"][s], s, int(c.get("mcc", 0)) if mode != 1 else 0,
                           c.get("gas_density", 0.0), c.get("sigma_el", 0.0),
                           c.get("sigma_iz0", 0.0), c.get("eps_th_ev", 0.0), c.get("qe", QE),
                           c.get("neutral_mass", 1.0), c.get("gas_temperature_ev", 0.0), k0, k1,
                           int(c.get("instance", 0)), self.step_count & 0xFFFFFFFF,
                           self.mesh.lx, self.mesh.ly, mode)

    def step(self, n_steps=1):
        for _ in range(n_steps):
            self._step_once()

    def _step_once(self):
        if self.implicit():
            # §3 DIPIC: predictor x~ = x + dt v (no kick, no collisions), then the field of the
            # predicted charge with the susceptibility, then the corrector v += dt a(x~),
            # x = x~ + dt^2 a(x~), and the collisions
            self._particle_pass(np.zeros((self.mesh.nleaf, 4, 2)), 1)
            _, _, E = self.fields()
            if self.diag is not None:
                self._diag_sample()
            self._particle_pass(E, 2)
        else:
            _, _, E = self.fields()
            if self.diag is not None:
                self._diag_sample()
            self._particle_pass(E, 0)
        self.step_count += 1

    def _particle_pass(self, E, mode):
        """One push pass of every species (mode: 0 leapfrog, 1 implicit predictor, 2 implicit
        corrector; or_push_mcc), then the §3.1 list update with the spawned pairs."""
        Eflat = np.ascontiguousarray(E.reshape(-1))
        results = []
        for s, sp in enumerate(self.species):
            if sp is None:
                results.append(None)
                continue
            n = sp.n
            new_leaf = np.empty(n, np.int64)
            spawn = np.zeros(n, np.uint8)
            sv = np.zeros(3 * n); svi = np.zeros(3 * n)
            p = self.push_params(s, mode)
            dec = np.empty(4 * n)
            e_part = None
            if self.shape():
                ex, ey = self.cic_field(sp)
                e_part = np.ascontiguousarray(np.stack([ex, ey], 1).reshape(-1))
            lib().or_push_mcc(C.byref(self.mesh._c), C.byref(p), _ptr(Eflat), n, _ptr(sp.x),
                              _ptr(sp.y), _ptr(sp.vx), _ptr(sp.vy), _ptr(sp.vz), _ptr(sp.id),
                              _ptr(sp.leaf), _ptr(new_leaf), _ptr(spawn), _ptr(sv), _ptr(svi),
                              _ptr(dec), _ptr(e_part))
            # the collision decisions of this step by particle id: (U0, P, U1 sigma_T, sigma_iz)
            if mode != 1:
                self.last_decisions[s] = (sp.id.copy(), dec.reshape(n, 4))
            results.append((new_leaf, spawn, sv.reshape(n, 3), svi.reshape(n, 3)))
        # spawned pairs (electrons only): ids next_id + 2*rank (electron), +1 (ion), rank =
        # position among the ionizing electrons in list order
        spawn_blocks = {}
        if self.species[0] is not None and results[0] is not None:
            new_leaf, spawn, sv, svi = results[0]
            par = np.nonzero(spawn)[0]
            k = par.size
            if k:
                base = self.next_id
                e_id = (base + 2 * np.arange(k)).astype(np.uint64)
                i_id = e_id + np.uint64(1)
                self.next_id = base + 2 * k
                sp = self.species[0]
                spawn_blocks[0] = (par, sp.x[par], sp.y[par], sv[par], sp.w[par], e_id, new_leaf[par])
                if len(self.species) > 1 and self.species[1] is not None:
                    spawn_blocks[1] = (par, sp.x[par], sp.y[par], svi[par], sp.w[par], i_id, new_leaf[par])
        for s, sp in enumerate(self.species):
            if sp is None:
                continue
            new_leaf = results[s][0]
            self.species[s] = self._rebin(sp, new_leaf, spawn_blocks.get(s))

    @staticmethod
    def _rebin(sp: Species, new_leaf, spawned):
        """§3.1 cell lists: stayers keep their order at the head of their list; particles
        entering a cell are appended in list order of their old position; pairs spawned
        this step are appended last, in the order of their parents."""
        n = sp.n
        alive = new_leaf >= 0
        idx = np.nonzero(alive)[0]
        leaf_new = new_leaf[idx]
        incoming = (leaf_new != sp.leaf[idx]).astype(np.int64)
        key3 = idx.astype(np.int64)
        parts = [sp.take(idx)]
        parts[0].leaf = leaf_new
        leaves = [leaf_new]; inc = [incoming]; k3 = [key3]
        if spawned is not None:
            par, x, y, v, w, ids, lf = spawned
            sp2 = Species(sp.q, sp.m, x.copy(), y.copy(), v[:, 0].copy(), v[:, 1].copy(),
                          v[:, 2].copy(), w.copy(), ids, lf.copy())
            keep = lf >= 0
            sp2 = sp2.take(np.nonzero(keep)[0])
            parts.append(sp2)
            leaves.append(sp2.leaf); inc.append(np.ones(sp2.n, np.int64))
            k3.append(n + par[keep].astype(np.int64))
        allp = _concat(parts)
        L = np.concatenate(leaves); I = np.concatenate(inc); K = np.concatenate(k3)
        order = np.lexsort((K, I, L))
        return allp.take(order)

    # -- read-out -----------------------------------------------------------------------
    def counts(self, s):
        sp = self.species[s]
        return np.bincount(sp.leaf, minlength=self.mesh.nleaf) if sp is not None else np.zeros(self.mesh.nleaf, np.int64)


def _concat(parts):
    p0 = parts[0]
    if len(parts) == 1:
        return p0
    cat = lambda name: np.concatenate([getattr(p, name) for p in parts])
    return Species(p0.q, p0.m, cat("x"), cat("y"), cat("vx"), cat("vy"), cat("vz"), cat("w"),
                   cat("id"), cat("leaf"))
