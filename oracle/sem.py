"""Plain FP64 spectral-element Burgers operators.  TEST INFRASTRUCTURE ONLY.

Follows Sec. 3 of arXiv:1806.01422 (Marin, Constantinescu, Smith):

* Eq. burgers23d:  du/dt = nu Lap(u) - (u . grad) u, periodic box [0, L)^d,
  u = (u_1..u_d) (d = 1 is the scalar 1D equation).
* Sec. 3.2 weak form with GLL collocation: diagonal mass, stiffness K = D^T M D,
  nonlinear term by collocation at the GLL points, affine element map with
  M_1 = (L/2) M and K_1 = (2/L) K.
* Sec. 3.3 tensor-product operators (eqs. rhsvec, jacvec, jactransvec): the
  Kronecker operators are applied one direction at a time (sum factorisation).

Notation used below (every symbol is a plain array):

* ``G = E*N`` unique periodic nodes per direction; global vectors have shape
  ``(d, G, .., G)`` with the LAST axis the x_0 (fastest) direction; component c
  is the velocity along physical direction x_c, i.e. array axis d-1-c.
* ``Q``: periodic scatter global -> element-local ("gather"), shape
  ``(d, E^d, n, .., n)``; ``Q^T``: sum of element contributions.
* ``B``: element-local diagonal GLL mass (h/2)^d w (x) w (x) w.
* ``M = Q^T B 1``: global diagonal mass.
* ``D_j``: collocation derivative along direction j, (2/h) Dhat.

Readings of the paper used here (it is garbled or silent on these points):

* sign: Eq. burgers23d is authoritative, so B du/dt = -nu K u - B (u . grad u);
* the 1D transpose printed with u o D^T[w] is read as D^T[u o w] (the 3D form
  D_j^T[u_j o w_i] of eq. jactransvec agrees);
* the "differential matrix" weights are carried by an explicit B.
"""
import numpy as np

from .gll import gll


class Grid:
    """Uniform periodic grid of E^d elements of order N on [0, L)^d (Sec. 3.2 affine map)."""

    def __init__(self, dim, E, N, nu, L=None):
        if dim not in (1, 2, 3):
            raise ValueError("dim must be 1, 2 or 3")
        self.d, self.E, self.N, self.nu = dim, E, N, float(nu)
        self.L = float(L if L is not None else (2 * np.pi if dim == 1 else 1.0))
        self.n = N + 1
        self.G = E * N
        self.h = self.L / E
        self.xi, self.w, self.Dh = gll(N)
        # element-local -> global index along one axis: (e*N + i) mod G
        e = np.arange(E)[:, None]
        i = np.arange(self.n)[None, :]
        self._idx1 = (e * N + i) % self.G
        self.nelem = E ** dim
        # B: element-local GLL mass (Sec. 3.2, M_1 = (L/2) M per direction with L = h),
        # shape (1, n, .., n) to broadcast over a flat element axis
        d = dim
        Bn = np.ones([1] + [self.n] * d)
        for p in range(d):
            shape = [1] * (1 + d)
            shape[1 + p] = self.n
            Bn = Bn * self.w.reshape(shape)
        self.B = (self.h / 2.0) ** d * Bn
        self.M = self.scatter_add(np.broadcast_to(self.B, self.local_shape()))

    # ----------------------------------------------------------------- layout
    # Elements are numbered e = ((e_{d-1} E) + ..) E + e_0 (e_0 along x_0, fastest);
    # element-local arrays have shape (nelem, n, .., n) with the node axes in
    # array order (x_{d-1}, .., x_0).
    def local_shape(self, nsel=None):
        return (self.nelem if nsel is None else nsel,) + (self.n,) * self.d

    def global_shape(self):
        return (self.G,) * self.d

    def ndof(self):
        return self.d * self.G ** self.d

    def coords(self):
        """Coordinates of the G unique nodes along one axis: e*h + (xi_i + 1) h / 2."""
        g = np.arange(self.G)
        e, i = g // self.N, g % self.N
        return e * self.h + (self.xi[i] + 1.0) * self.h / 2.0

    def elem_coords(self, elems):
        """Per-direction element coordinates (array order: e_{d-1}, .., e_0) of element ids."""
        elems = np.asarray(elems)
        out = []
        for p in range(self.d):
            out.append((elems // self.E ** (self.d - 1 - p)) % self.E)
        return out

    def _open_index(self, elems):
        ec = self.elem_coords(elems)
        idx = []
        for p in range(self.d):
            shape = [1] * (1 + self.d)
            shape[0] = len(ec[p])
            shape[1 + p] = self.n
            idx.append(self._idx1[ec[p]].reshape(shape))
        return tuple(idx)

    def gather(self, u, elems=None):
        """Q: global scalar field (G,..,G) -> element-local (nsel, n,..,n) (all elements by default)."""
        elems = np.arange(self.nelem) if elems is None else elems
        return u[self._open_index(elems)]

    def scatter_add(self, U):
        """Q^T: element-local (nelem, n,..,n) -> global, summing the copies of shared nodes."""
        out = np.zeros(self.global_shape())
        np.add.at(out, self._open_index(np.arange(self.nelem)), U)
        return out

    def node_axis(self, j):
        """Array axis of the element-local tile along physical direction x_j."""
        return 1 + (self.d - 1 - j)

    def apply_1d(self, A, X, axis):
        """Y[.., a, ..] = sum_m A[a, m] X[.., m, ..] along one axis (one Kronecker factor)."""
        return np.moveaxis(np.tensordot(A, X, axes=([1], [axis])), 0, axis)

    def grad(self, X, j):
        """D_j X = (2/h) Dhat along direction x_j of every element tile."""
        return (2.0 / self.h) * self.apply_1d(self.Dh, X, self.node_axis(j))

    def gradT(self, X, j):
        """D_j^T X = (2/h) Dhat^T along direction x_j."""
        return (2.0 / self.h) * self.apply_1d(self.Dh.T, X, self.node_axis(j))

    def gather_vec(self, u, elems=None):
        return np.stack([self.gather(u[c], elems) for c in range(self.d)])

    def scatter_vec(self, R):
        return np.stack([self.scatter_add(R[c]) for c in range(self.d)])

    # -------------------------------------------------------------- operators
    # Element-local residuals r_e (B-weighted, before the sum Q^T); each takes
    # element-local arrays of any number of elements.
    def local_rhs(self, U):
        """-nu sum_j D_j^T B D_j U_c - B sum_j U_j o D_j U_c  (eq. rhsvec, sign of Eq. burgers23d)."""
        d, B = self.d, self.B
        R = np.empty_like(U)
        for c in range(d):
            g = [self.grad(U[c], j) for j in range(d)]
            visc = sum(self.gradT(B * g[j], j) for j in range(d))
            adv = sum(U[j] * g[j] for j in range(d))
            R[c] = -self.nu * visc - B * adv
        return R

    def local_jac(self, U, W):
        """-nu sum_j D_j^T B D_j W_c - B sum_j (W_j o D_j U_c + U_j o D_j W_c)  (eq. jacvec)."""
        d, B = self.d, self.B
        R = np.empty_like(U)
        for c in range(d):
            gU = [self.grad(U[c], j) for j in range(d)]
            gW = [self.grad(W[c], j) for j in range(d)]
            visc = sum(self.gradT(B * gW[j], j) for j in range(d))
            adv = sum(W[j] * gU[j] + U[j] * gW[j] for j in range(d))
            R[c] = -self.nu * visc - B * adv
        return R

    def local_jacT(self, U, Z):
        """(L^T z)_l = -sum_j D_j^T( B o (nu D_j z_l + U_j o z_l) ) - B o sum_c z_c o D_l U_c  (eq. jactransvec)."""
        d, B = self.d, self.B
        R = np.empty_like(U)
        for l in range(d):
            flux = sum(self.gradT(B * (self.nu * self.grad(Z[l], j) + U[j] * Z[l]), j)
                       for j in range(d))
            react = sum(Z[c] * self.grad(U[c], l) for c in range(d))
            R[l] = -flux - B * react
        return R

    def rhs(self, u):
        """F(u) = M^-1 Q^T [ -nu sum_j D_j^T B D_j U_c - B sum_j U_j o D_j U_c ]  (eq. rhsvec).

        Eq. discrete3d gives M du/dt = nu K u - u . G u with K = sum_j D_j^T B D_j
        entering with the sign fixed by Eq. burgers23d (negative semidefinite
        viscous operator, minus the advection).
        """
        return self.scatter_vec(self.local_rhs(self.gather_vec(u))) / self.M

    def jac(self, u, w):
        """J(u) w = M^-1 Q^T [ -nu sum_j D_j^T B D_j W_c - B sum_j (W_j o D_j U_c + U_j o D_j W_c) ]  (eq. jacvec)."""
        return self.scatter_vec(self.local_jac(self.gather_vec(u), self.gather_vec(w))) / self.M

    def jacT(self, u, v):
        """J(u)^T v, the Euclidean transpose of ``jac`` (eq. jactransvec).

        With J = M^-1 Q^T L Q (L the element-local linear map of ``jac``), the
        transpose is Q^T L^T Q M^-1.  With z = Q M^-1 v:
          (L^T z)_l = -sum_j D_j^T( B o (nu D_j z_l + U_j o z_l) ) - B o sum_c z_c o D_l U_c.
        The three terms are eq. jactransvec's K_j^T[w_i], D_j^T[u_j o w_i] and
        w_j o D_i[u_j]; the 1D print u o D^T[w] is read as D^T[u o w].
        """
        return self.scatter_vec(self.local_jacT(self.gather_vec(u), self.gather_vec(v / self.M)))

    # ------------------------------------------- single-node evaluation (sampling)
    def sharing(self, node):
        """Elements sharing a global node (array-order index tuple) and its local index in each."""
        choices = []
        for p in range(self.d):
            g = node[p]
            e, i = g // self.N, g % self.N
            opts = [(e, i)]
            if i == 0:
                opts.append(((e - 1) % self.E, self.N))
            choices.append(opts)
        out = []
        for combo in np.ndindex(*[len(c) for c in choices]):
            ec = [choices[p][combo[p]] for p in range(self.d)]
            eid = 0
            for p in range(self.d):
                eid = eid * self.E + ec[p][0]
            out.append((eid, tuple(ec[p][1] for p in range(self.d))))
        return out

    def _at(self, local_fn, fields, nodes, divide_by_mass):
        vals = np.empty((self.d, len(nodes)))
        for k, node in enumerate(nodes):
            sh = self.sharing(node)
            elems = [e for e, _ in sh]
            R = local_fn(*[self.gather_vec(f, elems) for f in fields])
            for c in range(self.d):
                v = sum(R[(c, s) + loc] for s, (_, loc) in enumerate(sh))
                vals[c, k] = v / self.M[node] if divide_by_mass else v
        return vals

    def rhs_at(self, u, nodes):
        """F(u) at the listed global nodes only, from the elements sharing each node: shape (d, len(nodes))."""
        return self._at(self.local_rhs, [u], nodes, True)

    def jacT_at(self, u, v, nodes):
        """(J(u)^T v) at the listed global nodes only."""
        return self._at(self.local_jacT, [u, v / self.M], nodes, False)

    def jac_at(self, u, w, nodes):
        """(J(u) w) at the listed global nodes only."""
        return self._at(self.local_jac, [u, w], nodes, True)

    # -------------------------------------------------------------- objective
    def objective(self, u, u_obs):
        """J = 1/2 (u - u_obs)^T M (u - u_obs) and dJ/du = M (u - u_obs) (eqs. ourcost, initadj).

        The paper's misfit integral of (u(T) - u_d)^2 is discretised with the
        Galerkin inner product u^T M v (Sec. 4.1); the factor 1/2 follows the
        workload definition of the misfit.
        """
        r = u - u_obs
        lam = self.M[None] * r
        return 0.5 * float(np.sum(r * lam)), lam
