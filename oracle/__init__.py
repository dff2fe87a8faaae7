"""ctypes shim over the plain FP64 CPU oracle (``fmm_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  It shares
no code with the GPU library; numpy arrays in, numpy arrays out.

Complex coefficient vectors are numpy ``complex128`` arrays of length
``(p+1)**2``, index ``n*n + n + m`` for ``-n <= m <= n``.
"""
import ctypes
import numpy as np

from .build import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build())
        _declare(_lib)
    return _lib


_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_U64 = ctypes.POINTER(ctypes.c_uint64)
_I64 = ctypes.POINTER(ctypes.c_int64)
_i64 = ctypes.c_int64
_int = ctypes.c_int


def _declare(L):
    L.oracle_regular.argtypes = [_int, _D, _D]
    L.oracle_irregular.argtypes = [_int, _D, _D]
    L.oracle_direct.argtypes = [_i64, _D, _D, _i64, _D, _D, _D]
    L.oracle_p2m.argtypes = [_int, _D, _i64, _D, _D, _D]
    L.oracle_p2l.argtypes = [_int, _D, _i64, _D, _D, _D]
    L.oracle_m2m.argtypes = [_int, _D, _D, _D, _D]
    L.oracle_m2l.argtypes = [_int, _D, _D, _D, _D]
    L.oracle_l2l.argtypes = [_int, _D, _D, _D, _D]
    L.oracle_l2p.argtypes = [_int, _D, _D, _i64, _D, _D, _D]
    L.oracle_m2p.argtypes = [_int, _D, _D, _i64, _D, _D, _D]
    L.oracle_root_cube.argtypes = [_i64, _D, _D, _D]
    L.oracle_root_cube.restype = _int
    L.oracle_morton_keys.argtypes = [_i64, _D, _D, ctypes.c_double, _U64]
    L.oracle_tree_build.argtypes = [_i64, _D, _int, _int]
    L.oracle_tree_build.restype = ctypes.c_void_p
    L.oracle_tree_free.argtypes = [ctypes.c_void_p]
    L.oracle_tree_direct_wx.argtypes = [ctypes.c_void_p, _int]
    L.oracle_tree_sizes.argtypes = [ctypes.c_void_p, _I64]
    L.oracle_tree_geometry.argtypes = [ctypes.c_void_p, _D, _D]
    L.oracle_tree_export.argtypes = [ctypes.c_void_p, _U64, _I32, _I32, _U64] + [_I32] * 14
    L.oracle_fmm_eval.argtypes = [ctypes.c_void_p, _int, _D, _D, _D]
    L.oracle_num_threads.restype = _int
    L.oracle_dual_build.argtypes = [ctypes.c_void_p, ctypes.c_double]
    L.oracle_dual_build.restype = ctypes.c_void_p
    L.oracle_dual_free.argtypes = [ctypes.c_void_p]
    L.oracle_dual_sizes.argtypes = [ctypes.c_void_p, _I64]
    L.oracle_dual_export.argtypes = [ctypes.c_void_p, _I32, _I32, _I32, _I32, _D]
    L.oracle_dual_eval.argtypes = [ctypes.c_void_p, ctypes.c_void_p, _int, _D, _D, _D]
    dbl = ctypes.c_double
    L.oracle_sph_bessel.argtypes = [_int, dbl, _D, _D]
    L.oracle_sph_harmonics.argtypes = [_int, _D, _D]
    L.oracle_h_wave.argtypes = [_int, dbl, _D, _int, _D]
    L.oracle_gauss_legendre.argtypes = [_int, _D, _D]
    L.oracle_gaunt_size.argtypes = [_int]
    L.oracle_gaunt_size.restype = _i64
    L.oracle_gaunt_table.argtypes = [_int, _D]
    L.oracle_h_translate.argtypes = [_int, dbl, _D, _D, _int, _D, _D]
    L.oracle_h_direct.argtypes = [_i64, _D, _D, _i64, _D, dbl, _D]
    L.oracle_h_p2m.argtypes = [_int, dbl, _D, _i64, _D, _D, _D]
    L.oracle_h_p2l.argtypes = [_int, dbl, _D, _i64, _D, _D, _D]
    for f in ("oracle_h_m2m", "oracle_h_m2l", "oracle_h_l2l"):
        getattr(L, f).argtypes = [_int, dbl, _D, _D, _D, _D, _D]
    L.oracle_h_l2p.argtypes = [_int, dbl, _D, _D, _i64, _D, _D]
    L.oracle_h_m2p.argtypes = [_int, dbl, _D, _D, _i64, _D, _D]
    L.oracle_h_fmm_eval.argtypes = [ctypes.c_void_p, _int, dbl, _D, _D]


def _p(a, t=_D):
    return None if a is None else a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def ncoef(p):
    return (p + 1) * (p + 1)


def num_threads():
    return lib().oracle_num_threads()


def regular(p, x):
    out = np.zeros(ncoef(p), np.complex128)
    lib().oracle_regular(p, _p(_f64(x)), out.ctypes.data_as(_D))
    return out


def irregular(p, x):
    out = np.zeros(ncoef(p), np.complex128)
    lib().oracle_irregular(p, _p(_f64(x)), out.ctypes.data_as(_D))
    return out


def direct(src, q, tgt=None, grad=True):
    """phi (and grad) at ``tgt`` (default: the sources) from all sources;
    zero-distance pairs are skipped."""
    src = _f64(src).reshape(-1, 3)
    q = _f64(q)
    tgt = src if tgt is None else _f64(tgt).reshape(-1, 3)
    phi = np.zeros(len(tgt))
    g = np.zeros((len(tgt), 3)) if grad else None
    lib().oracle_direct(len(src), _p(src), _p(q), len(tgt), _p(tgt), _p(phi), _p(g))
    return (phi, g) if grad else phi


def p2m(p, c, xyz, q):
    M = np.zeros(ncoef(p), np.complex128)
    xyz = _f64(xyz).reshape(-1, 3)
    lib().oracle_p2m(p, _p(_f64(c)), len(xyz), _p(xyz), _p(_f64(q)), M.ctypes.data_as(_D))
    return M


def p2l(p, c, xyz, q):
    L = np.zeros(ncoef(p), np.complex128)
    xyz = _f64(xyz).reshape(-1, 3)
    lib().oracle_p2l(p, _p(_f64(c)), len(xyz), _p(xyz), _p(_f64(q)), L.ctypes.data_as(_D))
    return L


def _translate(fn, p, c_from, X, c_to):
    X = np.ascontiguousarray(X, np.complex128)
    out = np.zeros(ncoef(p), np.complex128)
    fn(p, _p(_f64(c_from)), X.ctypes.data_as(_D), _p(_f64(c_to)), out.ctypes.data_as(_D))
    return out


def m2m(p, c_child, M, c_parent):
    return _translate(lib().oracle_m2m, p, c_child, M, c_parent)


def m2l(p, c_src, M, c_tgt):
    return _translate(lib().oracle_m2l, p, c_src, M, c_tgt)


def l2l(p, c_parent, L, c_child):
    return _translate(lib().oracle_l2l, p, c_parent, L, c_child)


def _evaluate(fn, p, c, X, xyz):
    X = np.ascontiguousarray(X, np.complex128)
    xyz = _f64(xyz).reshape(-1, 3)
    phi = np.zeros(len(xyz))
    g = np.zeros((len(xyz), 3))
    fn(p, _p(_f64(c)), X.ctypes.data_as(_D), len(xyz), _p(xyz), _p(phi), _p(g))
    return phi, g


def l2p(p, c, L, xyz):
    return _evaluate(lib().oracle_l2p, p, c, L, xyz)


def m2p(p, c, M, xyz):
    return _evaluate(lib().oracle_m2p, p, c, M, xyz)


def root_cube(xyz):
    xyz = _f64(xyz).reshape(-1, 3)
    lo = np.zeros(3)
    D = np.zeros(1)
    rc = lib().oracle_root_cube(len(xyz), _p(xyz), _p(lo), _p(D))
    if rc != 0:
        raise ValueError("non-finite coordinate")
    return lo, float(D[0])


def morton_keys(xyz, lo, D):
    xyz = _f64(xyz).reshape(-1, 3)
    keys = np.zeros(len(xyz), np.uint64)
    lib().oracle_morton_keys(len(xyz), _p(xyz), _p(_f64(lo)), float(D), _p(keys, _U64))
    return keys


class Tree:
    """Adaptive octree + U/V/W/X lists built by the oracle."""

    FIELDS = ("keys", "perm", "level_offset", "box_key", "box_level", "box_first",
              "box_count", "box_parent", "box_child", "box_nchild", "u_off", "u_idx",
              "v_off", "v_idx", "w_off", "w_idx", "x_off", "x_idx")

    def __init__(self, xyz, leaf_size, max_depth=21, direct_wx=0):
        """``direct_wx`` > 0: W pairs of two leaves whose W leaf holds at most
        that many points go to the near field (oracle_tree_direct_wx)."""
        self.xyz = _f64(xyz).reshape(-1, 3)
        self.leaf_size = leaf_size
        self.max_depth = max_depth
        h = lib().oracle_tree_build(len(self.xyz), _p(self.xyz), leaf_size, max_depth)
        if not h:
            raise ValueError("oracle_tree_build rejected its arguments")
        self._h = h
        if direct_wx > 0:
            lib().oracle_tree_direct_wx(h, int(direct_wx))
        s = np.zeros(7, np.int64)
        lib().oracle_tree_sizes(h, _p(s, _I64))
        self.n, self.nboxes, self.nlevels = int(s[0]), int(s[1]), int(s[2])
        nu, nv, nw, nx = (int(v) for v in s[3:])
        lo = np.zeros(3)
        D = np.zeros(1)
        lib().oracle_tree_geometry(h, _p(lo), _p(D))
        self.lo, self.D = lo, float(D[0])
        n, nb = self.n, self.nboxes
        i32 = lambda k: np.zeros(k, np.int32)
        a = dict(keys=np.zeros(n, np.uint64), perm=i32(n), level_offset=i32(self.nlevels + 1),
                 box_key=np.zeros(nb, np.uint64), box_level=i32(nb), box_first=i32(nb),
                 box_count=i32(nb), box_parent=i32(nb), box_child=i32(nb), box_nchild=i32(nb),
                 u_off=i32(nb + 1), u_idx=i32(nu), v_off=i32(nb + 1), v_idx=i32(nv),
                 w_off=i32(nb + 1), w_idx=i32(nw), x_off=i32(nb + 1), x_idx=i32(nx))
        args = [_p(a[f], _U64 if a[f].dtype == np.uint64 else _I32) for f in self.FIELDS]
        lib().oracle_tree_export(h, *args)
        for f in self.FIELDS:
            setattr(self, f, a[f])

    def arrays(self):
        return {f: getattr(self, f) for f in self.FIELDS}

    def lst(self, name, b):
        off = getattr(self, name + "_off")
        return getattr(self, name + "_idx")[off[b]:off[b + 1]]

    def anchor(self, b):
        k = int(self.box_key[b])
        l = int(self.box_level[b])
        a = [0, 0, 0]
        for bit in range(l):
            for ax in range(3):
                a[ax] |= ((k >> (3 * bit + ax)) & 1) << bit
        return tuple(a)

    def side(self, b):
        return self.D * 2.0 ** (-int(self.box_level[b]))

    def center(self, b):
        a = self.anchor(b)
        s = self.side(b)
        return np.array([self.lo[i] + (a[i] + 0.5) * s for i in range(3)])

    def eval(self, p, q, grad=True):
        q = _f64(q)
        phi = np.zeros(self.n)
        g = np.zeros((self.n, 3)) if grad else None
        lib().oracle_fmm_eval(self._h, p, _p(q), _p(phi), _p(g))
        return (phi, g) if grad else phi

    def helmholtz_eval(self, p, kappa, q):
        """Helmholtz FMM mat-vec: complex q (input order) -> complex phi."""
        q = _c128(q)
        phi = np.zeros(self.n, np.complex128)
        lib().oracle_h_fmm_eval(self._h, p, float(kappa), _p(q), _p(phi))
        return phi

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.oracle_tree_free(h)
            self._h = None


class Dual:
    """Dual-tree traversal lists on an oracle ``Tree``: per target box its M2L
    sources (accepted by r_T + r_S < theta |c_T - c_S|) and its P2P source
    leaves, plus the cell radii."""

    def __init__(self, tree, theta):
        self.tree = tree
        self.theta = float(theta)
        h = lib().oracle_dual_build(tree._h, self.theta)
        self._h = h
        s = np.zeros(2, np.int64)
        lib().oracle_dual_sizes(h, _p(s, _I64))
        nb = tree.nboxes
        self.m2l_off = np.zeros(nb + 1, np.int32)
        self.m2l_idx = np.zeros(int(s[0]), np.int32)
        self.p2p_off = np.zeros(nb + 1, np.int32)
        self.p2p_idx = np.zeros(int(s[1]), np.int32)
        self.radius = np.zeros(nb)
        lib().oracle_dual_export(h, _p(self.m2l_off, _I32), _p(self.m2l_idx, _I32),
                                 _p(self.p2p_off, _I32), _p(self.p2p_idx, _I32),
                                 _p(self.radius))

    def lst(self, name, b):
        off = getattr(self, name + "_off")
        return getattr(self, name + "_idx")[off[b]:off[b + 1]]

    def eval(self, p, q, grad=True):
        q = _f64(q)
        phi = np.zeros(self.tree.n)
        g = np.zeros((self.tree.n, 3)) if grad else None
        lib().oracle_dual_eval(self.tree._h, self._h, p, _p(q), _p(phi), _p(g))
        return (phi, g) if grad else phi

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.oracle_dual_free(h)
            self._h = None


# ---------------------------------------------------------------- Helmholtz
# Kernel e^{i kappa r}/r; complex arrays are numpy complex128.

def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def sph_bessel(nmax, x):
    """(j_0..j_nmax, y_0..y_nmax) at x > 0."""
    j = np.zeros(nmax + 1)
    y = np.zeros(nmax + 1)
    lib().oracle_sph_bessel(nmax, float(x), _p(j), _p(y))
    return j, y


def sph_harmonics(p, x):
    Y = np.zeros(ncoef(p), np.complex128)
    lib().oracle_sph_harmonics(p, _p(_f64(x)), _p(Y))
    return Y


def h_wave(p, kappa, x, singular):
    X = np.zeros(ncoef(p), np.complex128)
    lib().oracle_h_wave(p, float(kappa), _p(_f64(x)), int(bool(singular)), _p(X))
    return X


def gauss_legendre(n):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().oracle_gauss_legendre(n, _p(x), _p(w))
    return x, w


def gaunt_table(p):
    G = np.zeros(lib().oracle_gaunt_size(p))
    lib().oracle_gaunt_table(p, _p(G))
    return G


def gaunt(G, p, n, m, n2, m2, l):
    """G(n,m; n2,m2; l) from a table of gaunt_table(p)."""
    l0 = abs(n - n2)
    if l < l0 or l > n + n2 or (l - l0) % 2 or abs(m - m2) > l:
        return 0.0
    nc = ncoef(p)
    return G[((n * n + n + m) * nc + n2 * n2 + n2 + m2) * (p + 1) + (l - l0) // 2]


def h_translate(p, kappa, G, t, singular, X_in):
    out = np.zeros(ncoef(p), np.complex128)
    lib().oracle_h_translate(p, float(kappa), _p(G), _p(_f64(t)), int(bool(singular)),
                             _p(_c128(X_in)), _p(out))
    return out


def h_direct(src, q, kappa, tgt=None):
    src = _f64(src).reshape(-1, 3)
    tgt = src if tgt is None else _f64(tgt).reshape(-1, 3)
    q = _c128(q)
    phi = np.zeros(len(tgt), np.complex128)
    lib().oracle_h_direct(len(src), _p(src), _p(q), len(tgt), _p(tgt), float(kappa), _p(phi))
    return phi


def h_p2m(p, kappa, c, xyz, q):
    xyz = _f64(xyz).reshape(-1, 3)
    M = np.zeros(ncoef(p), np.complex128)
    lib().oracle_h_p2m(p, float(kappa), _p(_f64(c)), len(xyz), _p(xyz), _p(_c128(q)), _p(M))
    return M


def h_p2l(p, kappa, c, xyz, q):
    xyz = _f64(xyz).reshape(-1, 3)
    L = np.zeros(ncoef(p), np.complex128)
    lib().oracle_h_p2l(p, float(kappa), _p(_f64(c)), len(xyz), _p(xyz), _p(_c128(q)), _p(L))
    return L


def _h_translate3(fn, p, kappa, G, c_from, X, c_to):
    out = np.zeros(ncoef(p), np.complex128)
    getattr(lib(), fn)(p, float(kappa), _p(G), _p(_f64(c_from)), _p(_c128(X)), _p(_f64(c_to)),
                       _p(out))
    return out


def h_m2m(p, kappa, G, c_child, M, c_parent):
    return _h_translate3("oracle_h_m2m", p, kappa, G, c_child, M, c_parent)


def h_m2l(p, kappa, G, c_src, M, c_tgt):
    return _h_translate3("oracle_h_m2l", p, kappa, G, c_src, M, c_tgt)


def h_l2l(p, kappa, G, c_parent, L, c_child):
    return _h_translate3("oracle_h_l2l", p, kappa, G, c_parent, L, c_child)


def h_l2p(p, kappa, c, L, xyz):
    xyz = _f64(xyz).reshape(-1, 3)
    phi = np.zeros(len(xyz), np.complex128)
    lib().oracle_h_l2p(p, float(kappa), _p(_f64(c)), _p(_c128(L)), len(xyz), _p(xyz), _p(phi))
    return phi


def h_m2p(p, kappa, c, M, xyz):
    xyz = _f64(xyz).reshape(-1, 3)
    phi = np.zeros(len(xyz), np.complex128)
    lib().oracle_h_m2p(p, float(kappa), _p(_f64(c)), _p(_c128(M)), len(xyz), _p(xyz), _p(phi))
    return phi
