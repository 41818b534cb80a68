"""Iterative charted refinement (ICR) on a 2-D log-radial chart (oracle; test
infrastructure only).

Sec. "Gaussian Processes" (ICR paragraph): a GP on an arbitrarily deformed space
built by refining a coarse sample level by level from nearest-neighbour
relations on coarsenings of the chart.  The paper gives no equations; the
reading used throughout this project:

* Chart: level l has n_l = n0 2^l points per axis at chart coordinates
  u = (i + 1/2)/n_l, v = (j + 1/2)/n_l, mapped to the plane by
  r = r_min (r_max / r_min)^u, phi = 2 pi v, position (r cos phi, r sin phi).
  Coarse index i has the fine children 2i and 2i + 1 on each axis.
* Kernel: Matern-3/2, k(d) = var (1 + sqrt(3) d / rho) exp(-sqrt(3) d / rho),
  on Euclidean distance.
* Level 0: s_0 = L_K0 xi_0 with L_K0 the lower Cholesky factor of the kernel
  matrix of all n0^2 level-0 points (C order).
* Refinement of coarse pixel (i, j): its neighbourhood is the 3 radial rows
  w(i), w(i)+1, w(i)+2 with w(i) = clip(i - 1, 0, n_c - 3) (a window clamped at
  the radial edges) times the angular columns j-1, j, j+1 modulo n_c (periodic),
  ordered row-major; its four children (2i+a, 2j+b), a, b in {0, 1}, ordered
  2a + b.  With K_cc (9x9), K_fc (4x9), K_ff (4x4) the kernel blocks,
      R = K_fc K_cc^-1,  D = K_ff - K_fc K_cc^-1 K_cf,  L_D = chol(D),
      s_children = R s_neighbourhood + L_D xi_children.
  Rotation by 2 pi / n_c maps the chart onto itself, so R and L_D depend only on
  the level and the radial row i; they are built for column j = 0.
* Latent layout: xi_0, xi_1, ..., xi_L concatenated, each n_l x n_l in C order.
* ICR metric: Gaussian likelihood with noise std sigma on s of the finest level
  (identity response): M v = v + L^T L v / sigma^2.
"""
import numpy as np


class ICRChart:
    def __init__(self, n0=8, n_levels=7, r_min=0.1, r_max=1.0, rho=0.1, var=1.0):
        if n0 < 3:
            raise ValueError("n0 must be >= 3 for the 3x3 neighbourhood")
        self.n0 = int(n0)
        self.n_levels = int(n_levels)
        self.r_min = float(r_min)
        self.r_max = float(r_max)
        self.rho = float(rho)
        self.var = float(var)
        self.sizes = [self.n0 * 2 ** l for l in range(self.n_levels + 1)]
        self.offsets = np.concatenate([[0], np.cumsum([n * n for n in self.sizes])])
        self.latent_size = int(self.offsets[-1])
        self._L0 = None
        self._mats = {}

    # geometry -------------------------------------------------------------
    def position(self, level, i, j):
        n = self.sizes[level]
        u = (np.asarray(i, dtype=np.float64) + 0.5) / n
        v = (np.asarray(j, dtype=np.float64) + 0.5) / n
        r = self.r_min * (self.r_max / self.r_min) ** u
        phi = 2.0 * np.pi * v
        return np.stack([r * np.cos(phi), r * np.sin(phi)], axis=-1)

    def kernel(self, d):
        t = np.sqrt(3.0) * d / self.rho
        return self.var * (1.0 + t) * np.exp(-t)

    def kmat(self, pa, pb):
        d = np.sqrt(np.sum((pa[:, None, :] - pb[None, :, :]) ** 2, axis=-1))
        return self.kernel(d)

    def window(self, level, i):
        return int(np.clip(i - 1, 0, self.sizes[level] - 3))

    # matrices -------------------------------------------------------------
    def L0(self):
        if self._L0 is None:
            n = self.n0
            # all level-0 points, C order
            ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
            p = self.position(0, ii.ravel(), jj.ravel())
            K = self.kmat(p, p)
            try:
                self._L0 = np.linalg.cholesky(K)
            except np.linalg.LinAlgError:
                self._L0 = np.linalg.cholesky(K + 1e-10 * self.var * np.eye(n * n))
        return self._L0

    def coarse_fine_points(self, level, i):
        """Neighbourhood (9) and children (4) positions of coarse (level, i, j=0)."""
        nc = self.sizes[level]
        w = self.window(level, i)
        ci = np.array([w + a for a in range(3) for _ in range(3)])
        cj = np.array([(b - 1) % nc for _ in range(3) for b in range(3)])
        fi = np.array([2 * i + a for a in range(2) for _ in range(2)])
        fj = np.array([b for _ in range(2) for b in range(2)])
        return self.position(level, ci, cj), self.position(level + 1, fi, fj)

    def matrices(self, level):
        """R (n_c, 4, 9) and L_D (n_c, 4, 4) for refining ``level`` -> ``level+1``."""
        if level not in self._mats:
            nc = self.sizes[level]
            R = np.zeros((nc, 4, 9))
            LD = np.zeros((nc, 4, 4))
            for i in range(nc):
                pc, pf = self.coarse_fine_points(level, i)
                Kcc = self.kmat(pc, pc)
                Kfc = self.kmat(pf, pc)
                Kff = self.kmat(pf, pf)
                Ri = np.linalg.solve(Kcc, Kfc.T).T
                D = Kff - Ri @ Kfc.T
                R[i] = Ri
                LD[i] = np.linalg.cholesky(D)
            self._mats[level] = (R, LD)
        return self._mats[level]

    # latent helpers -------------------------------------------------------
    def split(self, xi):
        xi = np.asarray(xi, dtype=np.float64)
        assert xi.shape == (self.latent_size,)
        return [xi[self.offsets[l]:self.offsets[l + 1]].reshape(n, n)
                for l, n in enumerate(self.sizes)]

    def _nbhd_index(self, level):
        nc = self.sizes[level]
        w = np.clip(np.arange(nc) - 1, 0, nc - 3)
        rows = w[:, None] + np.arange(3)[None, :]                     # (nc, 3)
        cols = (np.arange(nc)[:, None] + np.arange(-1, 2)[None, :]) % nc  # (nc, 3)
        RI = np.broadcast_to(rows[:, None, :, None], (nc, nc, 3, 3)).reshape(nc, nc, 9)
        CJ = np.broadcast_to(cols[None, :, None, :], (nc, nc, 3, 3)).reshape(nc, nc, 9)
        return RI, CJ

    @staticmethod
    def _blocks(f):
        """(2n, 2n) fine array -> (n, n, 4) child blocks ordered 2a + b."""
        n2 = f.shape[0]
        return f.reshape(n2 // 2, 2, n2 // 2, 2).transpose(0, 2, 1, 3).reshape(n2 // 2, n2 // 2, 4)

    @staticmethod
    def _unblocks(b):
        n = b.shape[0]
        return b.reshape(n, n, 2, 2).transpose(0, 2, 1, 3).reshape(2 * n, 2 * n)

    # model ----------------------------------------------------------------
    def refine(self, level, s_c, xi_f):
        R, LD = self.matrices(level)
        RI, CJ = self._nbhd_index(level)
        nbh = s_c[RI, CJ]                                  # (nc, nc, 9)
        blk = (np.einsum("ikn,ijn->ijk", R, nbh)
               + np.einsum("ikm,ijm->ijk", LD, self._blocks(xi_f)))
        return self._unblocks(blk)

    def forward(self, xi, return_levels=False):
        xs = self.split(xi)
        s = (self.L0() @ xs[0].ravel()).reshape(self.n0, self.n0)
        levels = [s]
        for l in range(self.n_levels):
            s = self.refine(l, s, xs[l + 1])
            levels.append(s)
        return levels if return_levels else s

    def jvp(self, v):
        return self.forward(v)   # the map xi -> s is linear

    def vjp(self, g):
        g = np.asarray(g, dtype=np.float64).reshape(self.sizes[-1], self.sizes[-1])
        out = [None] * (self.n_levels + 1)
        for l in range(self.n_levels - 1, -1, -1):
            R, LD = self.matrices(l)
            RI, CJ = self._nbhd_index(l)
            G = self._blocks(g)                                   # (nc, nc, 4)
            out[l + 1] = self._unblocks(np.einsum("ikm,ijk->ijm", LD, G))
            contrib = np.einsum("ikn,ijk->ijn", R, G)             # (nc, nc, 9)
            nc = self.sizes[l]
            gc = np.zeros((nc, nc))
            np.add.at(gc, (RI, CJ), contrib)
            g = gc
        out[0] = (self.L0().T @ g.ravel()).reshape(self.n0, self.n0)
        return np.concatenate([o.ravel() for o in out])

    def metric_apply(self, v, sigma=0.1):
        v = np.asarray(v, dtype=np.float64)
        return v + self.vjp(self.forward(v)) / (sigma * sigma)
