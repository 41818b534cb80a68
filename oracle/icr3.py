"""Iterative charted refinement on a 3-D chart (oracle; test infrastructure only).

Sec. "Gaussian Processes" (ICR paragraph): the refinement scheme of
``oracle.icr`` on a three-dimensional chart, the setting of the tomography
application the paper mentions.  Reading used throughout this project:

* Chart: level l has n_l = n0 2^l points per axis at chart coordinates
  u = (i + 1/2)/n_l, v = (j + 1/2)/n_l, t = (k + 1/2)/n_l, mapped to a
  spherical log-radial shell: r = r_min (r_max / r_min)^u, polar angle
  theta = pi v, azimuth phi = 2 pi t, position
  r (sin theta cos phi, sin theta sin phi, cos theta).  Coarse index i has the
  fine children 2i and 2i + 1 on each axis.
* Kernel: Matern-3/2 on Euclidean distance, as in 2-D.
* Level 0: s_0 = L_K0 xi_0 with L_K0 = chol of the kernel matrix of all n0^3
  level-0 points (C order).
* Refinement of coarse voxel (i, j, k): its neighbourhood is the radial rows
  w(i)..w(i)+2 and the polar rows w(j)..w(j)+2, w(x) = clip(x - 1, 0, n_c - 3)
  (windows clamped at the chart's edges), times the azimuthal columns k-1, k,
  k+1 modulo n_c (periodic), ordered 9a + 3b + c; its eight children
  (2i+a, 2j+b, 2k+c) are ordered 4a + 2b + c.  R = K_fc K_cc^-1 (8 x 27),
  D = K_ff - R K_cf, L_D = chol(D);  s_children = R s_nbhd + L_D xi_children.
  Rotation about the polar axis maps the chart onto itself, so R and L_D
  depend on the level, the radial row i and the polar row j; they are built
  for k = 0.
* Latent layout: xi_0, ..., xi_L, each n_l^3 in C order.
* Metric: Gaussian likelihood with std sigma on the finest level (identity
  response): M v = v + L^T L v / sigma^2.
"""
import numpy as np


class ICRChart3D:
    def __init__(self, n0=4, n_levels=3, r_min=0.1, r_max=1.0, rho=0.3, var=1.0):
        if n0 < 3:
            raise ValueError("n0 must be >= 3 for the 3x3x3 neighbourhood")
        self.n0 = int(n0)
        self.n_levels = int(n_levels)
        self.r_min = float(r_min)
        self.r_max = float(r_max)
        self.rho = float(rho)
        self.var = float(var)
        self.sizes = [self.n0 * 2 ** l for l in range(self.n_levels + 1)]
        self.offsets = np.concatenate([[0], np.cumsum([n ** 3 for n in self.sizes])])
        self.latent_size = int(self.offsets[-1])
        self._L0 = None
        self._mats = {}

    # geometry -------------------------------------------------------------
    def position(self, level, i, j, k):
        n = self.sizes[level]
        u = (np.asarray(i, dtype=np.float64) + 0.5) / n
        v = (np.asarray(j, dtype=np.float64) + 0.5) / n
        t = (np.asarray(k, dtype=np.float64) + 0.5) / n
        r = self.r_min * (self.r_max / self.r_min) ** u
        th = np.pi * v
        ph = 2.0 * np.pi * t
        return np.stack([r * np.sin(th) * np.cos(ph), r * np.sin(th) * np.sin(ph), r * np.cos(th)], axis=-1)

    def kernel(self, d):
        x = np.sqrt(3.0) * d / self.rho
        return self.var * (1.0 + x) * np.exp(-x)

    def kmat(self, pa, pb):
        d = np.sqrt(np.sum((pa[:, None, :] - pb[None, :, :]) ** 2, axis=-1))
        return self.kernel(d)

    def window(self, level, i):
        return int(np.clip(i - 1, 0, self.sizes[level] - 3))

    # matrices -------------------------------------------------------------
    def L0(self):
        if self._L0 is None:
            n = self.n0
            ii, jj, kk = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
            p = self.position(0, ii.ravel(), jj.ravel(), kk.ravel())
            K = self.kmat(p, p)
            try:
                self._L0 = np.linalg.cholesky(K)
            except np.linalg.LinAlgError:
                self._L0 = np.linalg.cholesky(K + 1e-10 * self.var * np.eye(n ** 3))
        return self._L0

    def coarse_fine_points(self, level, i, j):
        """Neighbourhood (27) and children (8) positions of coarse (level, i, j, k=0)."""
        nc = self.sizes[level]
        wi, wj = self.window(level, i), self.window(level, j)
        nb = [(wi + a, wj + b, (c - 1) % nc) for a in range(3) for b in range(3) for c in range(3)]
        ch = [(2 * i + a, 2 * j + b, c) for a in range(2) for b in range(2) for c in range(2)]
        pc = self.position(level, *np.array(nb).T)
        pf = self.position(level + 1, *np.array(ch).T)
        return pc, pf

    def matrices(self, level):
        """R (n_c, n_c, 8, 27) and L_D (n_c, n_c, 8, 8) for level -> level + 1."""
        if level not in self._mats:
            nc = self.sizes[level]
            R = np.zeros((nc, nc, 8, 27))
            LD = np.zeros((nc, nc, 8, 8))
            for i in range(nc):
                for j in range(nc):
                    pc, pf = self.coarse_fine_points(level, i, j)
                    Kcc = self.kmat(pc, pc)
                    Kfc = self.kmat(pf, pc)
                    Kff = self.kmat(pf, pf)
                    Rij = np.linalg.solve(Kcc, Kfc.T).T
                    R[i, j] = Rij
                    LD[i, j] = np.linalg.cholesky(Kff - Rij @ Kfc.T)
            self._mats[level] = (R, LD)
        return self._mats[level]

    # latent helpers -------------------------------------------------------
    def split(self, xi):
        xi = np.asarray(xi, dtype=np.float64)
        assert xi.shape == (self.latent_size,)
        return [xi[self.offsets[l]:self.offsets[l + 1]].reshape(n, n, n) for l, n in enumerate(self.sizes)]

    def _nbhd_index(self, level):
        nc = self.sizes[level]
        w = np.clip(np.arange(nc) - 1, 0, nc - 3)
        rows = w[:, None] + np.arange(3)[None, :]                           # (nc, 3)
        cols = (np.arange(nc)[:, None] + np.arange(-1, 2)[None, :]) % nc    # (nc, 3)
        I = np.broadcast_to(rows[:, None, None, :, None, None], (nc, nc, nc, 3, 3, 3)).reshape(nc, nc, nc, 27)
        J = np.broadcast_to(rows[None, :, None, None, :, None], (nc, nc, nc, 3, 3, 3)).reshape(nc, nc, nc, 27)
        K = np.broadcast_to(cols[None, None, :, None, None, :], (nc, nc, nc, 3, 3, 3)).reshape(nc, nc, nc, 27)
        return I, J, K

    @staticmethod
    def _blocks(f):
        """(2n)^3 fine array -> (n, n, n, 8) child blocks ordered 4a + 2b + c."""
        n = f.shape[0] // 2
        return f.reshape(n, 2, n, 2, n, 2).transpose(0, 2, 4, 1, 3, 5).reshape(n, n, n, 8)

    @staticmethod
    def _unblocks(b):
        n = b.shape[0]
        return b.reshape(n, n, n, 2, 2, 2).transpose(0, 3, 1, 4, 2, 5).reshape(2 * n, 2 * n, 2 * n)

    # model ----------------------------------------------------------------
    def refine(self, level, s_c, xi_f):
        R, LD = self.matrices(level)
        I, J, K = self._nbhd_index(level)
        nbh = s_c[I, J, K]                                               # (nc, nc, nc, 27)
        blk = (np.einsum("ijmn,ijkn->ijkm", R, nbh)
               + np.einsum("ijmq,ijkq->ijkm", LD, self._blocks(xi_f)))
        return self._unblocks(blk)

    def forward(self, xi, return_levels=False):
        xs = self.split(xi)
        s = (self.L0() @ xs[0].ravel()).reshape(self.n0, self.n0, self.n0)
        levels = [s]
        for l in range(self.n_levels):
            s = self.refine(l, s, xs[l + 1])
            levels.append(s)
        return levels if return_levels else s

    def jvp(self, v):
        return self.forward(v)   # the map xi -> s is linear

    def vjp(self, g):
        n = self.sizes[-1]
        g = np.asarray(g, dtype=np.float64).reshape(n, n, n)
        out = [None] * (self.n_levels + 1)
        for l in range(self.n_levels - 1, -1, -1):
            R, LD = self.matrices(l)
            I, J, K = self._nbhd_index(l)
            G = self._blocks(g)                                           # (nc, nc, nc, 8)
            out[l + 1] = self._unblocks(np.einsum("ijmq,ijkm->ijkq", LD, G))
            contrib = np.einsum("ijmn,ijkm->ijkn", R, G)                  # (nc, nc, nc, 27)
            nc = self.sizes[l]
            gc = np.zeros((nc, nc, nc))
            np.add.at(gc, (I, J, K), contrib)
            g = gc
        out[0] = (self.L0().T @ g.ravel()).reshape(self.n0, self.n0, self.n0)
        return np.concatenate([o.ravel() for o in out])

    def metric_apply(self, v, sigma=0.1):
        v = np.asarray(v, dtype=np.float64)
        return v + self.vjp(self.forward(v)) / (sigma * sigma)
