"""Seeded synthetic inputs shared by the CPU oracle, the tests and the benchmark.

This module only *draws* inputs; it holds none of the contraction, H_eff,
Lanczos or theta arithmetic.  Every generator is deterministic in its seed
(numpy PCG64 via ``default_rng``), so the oracle and the CUDA path receive
bitwise-identical operands.

Workload recipes (there is no public dataset for this path):

* Dense two-site DMRG effective Hamiltonian, spin-1/2 Heisenberg chain:
  psi[a', t1, t2, b'] (chi x 2 x 2 x chi), L[a, w, a'] and R[b, w, b']
  (chi x 5 x chi) i.i.d. N(0,1); L and R are symmetrised channel-wise as
  L_w <- (L_w + L_{sigma(w)}^T)/2 with sigma swapping the S+ and S- channels
  (1 <-> 2), which makes the effective Hamiltonian a symmetric matrix so a
  Lanczos eigensolve on it is well posed.
* MPO: the standard lower-triangular 5x5 Heisenberg MPO, W[wl, wr, s, t]
  with s the bra (output) and t the ket (input) physical index.
* U(1) block-sparse variant: charge sectors q in [-15, 15], sector dims
  proportional to exp(-q^2 / (2 sigma^2)) with sigma = 5, apportioned by
  largest remainder (each sector at least 1) to sum to the total bond
  dimension.  Physical charges c(up) = +1, c(down) = -1; MPO channel charges
  Delta = [0, +2, -2, 0, 0] so that W[wl, wr, s, t] != 0 only when
  c(s) - c(t) = Delta[wl] - Delta[wr].  Blocks are N(0,1) float32.
* Batched TEBD theta: bond dims chi_i ~ U{16..512}; A_i[chi, 2, chi] and
  B_i[chi, 2, chi] complex64 with N(0,1) real and imaginary parts; each gate
  G_i[s1, s2, t1, t2] a Haar-random 4x4 unitary (QR of a complex Gaussian
  with the phases of R's diagonal divided out, Mezzadri 2007).
"""
from __future__ import annotations

import numpy as np

DEFAULT_SEED = 20251223

# ---------------------------------------------------------------------------
# Spin-1/2 operators in the basis (up, down) = (0, 1); op[s, t] = <s|op|t>.
# ---------------------------------------------------------------------------
SZ = np.array([[0.5, 0.0], [0.0, -0.5]])
SP = np.array([[0.0, 1.0], [0.0, 0.0]])   # S+ |down> = |up>
SM = np.array([[0.0, 0.0], [1.0, 0.0]])   # S- |up>   = |down>
ID2 = np.eye(2)

# U(1) charges (units of 2 S^z) of the physical states and MPO channels.
PHYS_CHARGE = np.array([+1, -1])
MPO_CHANNEL_CHARGE = np.array([0, +2, -2, 0, 0])
# sigma: channel map under operator transposition (S+ <-> S-).
MPO_SIGMA = np.array([0, 2, 1, 3, 4])


def heisenberg_mpo(J: float = 1.0) -> np.ndarray:
    """Lower-triangular Heisenberg MPO W[wl, wr, s, t], Dw = 5, d = 2.

    H = J sum_i [ (S+_i S-_{i+1} + S-_i S+_{i+1})/2 + Sz_i Sz_{i+1} ];
    the left boundary vector selects wl = 4 and the right one wr = 0.
    """
    W = np.zeros((5, 5, 2, 2))
    W[0, 0] = ID2
    W[1, 0] = SP
    W[2, 0] = SM
    W[3, 0] = SZ
    W[4, 1] = 0.5 * J * SM
    W[4, 2] = 0.5 * J * SP
    W[4, 3] = J * SZ
    W[4, 4] = ID2
    return W


def symmetrise_env(E: np.ndarray) -> np.ndarray:
    """E[x, w, x'] -> (E_w + E_{sigma(w)}^T)/2 channel-wise (see module doc)."""
    Et = np.transpose(E, (2, 1, 0))[:, MPO_SIGMA, :]
    return 0.5 * (E + Et)


def dense_heff_inputs(chi: int, seed: int = DEFAULT_SEED, chi_r: int | None = None,
                      symmetrise: bool = True):
    """psi[chi, 2, 2, chi_r], L[chi, 5, chi], R[chi_r, 5, chi_r], W[5, 5, 2, 2] (float64)."""
    chi_r = chi if chi_r is None else chi_r
    rng = np.random.default_rng(seed)
    psi = rng.standard_normal((chi, 2, 2, chi_r))
    L = rng.standard_normal((chi, 5, chi))
    R = rng.standard_normal((chi_r, 5, chi_r))
    if symmetrise:
        L = symmetrise_env(L)
        R = symmetrise_env(R)
    return psi, np.ascontiguousarray(L), np.ascontiguousarray(R), heisenberg_mpo(1.0)


def random_tensor(shape, seed: int, dtype=np.float64) -> np.ndarray:
    """A tensor of i.i.d. N(0,1) entries (complex: N(0,1) real and imaginary parts)."""
    rng = np.random.default_rng(seed)
    dtype = np.dtype(dtype)
    if dtype.kind == "c":
        re = rng.standard_normal(shape)
        im = rng.standard_normal(shape)
        return (re + 1j * im).astype(dtype)
    return rng.standard_normal(shape).astype(dtype)


# ---------------------------------------------------------------------------
# U(1) block-sparse inputs
# ---------------------------------------------------------------------------
def sector_dims(total: int = 2048, qmax: int = 15, sigma: float = 5.0) -> np.ndarray:
    """Sector dims for q = -qmax..qmax, proportional to a Gaussian, summing to ``total``.

    Largest-remainder apportionment with a floor of 1 per sector; ties in the
    remainder are broken towards smaller |q| (then smaller q) so the result is
    deterministic and symmetric.
    """
    q = np.arange(-qmax, qmax + 1)
    wgt = np.exp(-q.astype(np.float64) ** 2 / (2.0 * sigma ** 2))
    nsec = len(q)
    if total < nsec:
        raise ValueError("total bond dimension smaller than the number of sectors")
    free = total - nsec                      # one state per sector is reserved
    share = free * wgt / wgt.sum()
    base = np.floor(share).astype(np.int64)
    rem = share - base
    left = free - int(base.sum())
    order = sorted(range(nsec), key=lambda i: (-rem[i], abs(q[i]), q[i]))
    for i in order[:left]:
        base[i] += 1
    dims = base + 1
    assert int(dims.sum()) == total
    return dims


def sector_offsets(dims: np.ndarray) -> np.ndarray:
    return np.concatenate([[0], np.cumsum(dims)[:-1]]).astype(np.int64)


def blocksparse_structure(dims: np.ndarray, qmax: int = 15):
    """Allowed blocks of psi, L and R under the U(1) rules in the module doc.

    Returns dict with lists of keys:
      psi: (ia', t1, t2, ib')  with q_b' = q_a' + c(t1) + c(t2)
      L:   (ia, w, ia')        with q_a  = q_a' - Delta[w]
      R:   (ib, w, ib')        with q_b  = q_b' - Delta[w]
    where ia etc. are sector indices (q = index - qmax).
    """
    nsec = len(dims)

    def idx(qv):
        i = qv + qmax
        return i if 0 <= i < nsec else None

    psi, Lb, Rb = [], [], []
    for ia in range(nsec):
        qa = ia - qmax
        for t1 in range(2):
            for t2 in range(2):
                ib = idx(qa + PHYS_CHARGE[t1] + PHYS_CHARGE[t2])
                if ib is not None:
                    psi.append((ia, t1, t2, ib))
        for w in range(5):
            j = idx(qa + MPO_CHANNEL_CHARGE[w])    # q_a' = q_a + Delta[w]
            if j is not None:
                Lb.append((ia, w, j))
                Rb.append((ia, w, j))
    return {"psi": psi, "L": Lb, "R": Rb}


def blocksparse_inputs(total: int = 2048, seed: int = DEFAULT_SEED, qmax: int = 15,
                       sigma: float = 5.0):
    """Block-sparse psi, L, R (float32 blocks, N(0,1)) and the Heisenberg MPO.

    Blocks are drawn in the order of ``blocksparse_structure`` (psi, then L,
    then R), each as a C-contiguous float32 array of its block shape.
    """
    dims = sector_dims(total, qmax, sigma)
    st = blocksparse_structure(dims, qmax)
    rng = np.random.default_rng(seed)
    psi = {k: rng.standard_normal((dims[k[0]], dims[k[3]])).astype(np.float32) for k in st["psi"]}
    L = {k: rng.standard_normal((dims[k[0]], dims[k[2]])).astype(np.float32) for k in st["L"]}
    R = {k: rng.standard_normal((dims[k[0]], dims[k[2]])).astype(np.float32) for k in st["R"]}
    return {"dims": dims, "qmax": qmax, "psi": psi, "L": L, "R": R, "W": heisenberg_mpo(1.0)}


# ---------------------------------------------------------------------------
# Batched TEBD inputs
# ---------------------------------------------------------------------------
def haar_unitary(n: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-random n x n unitary: QR of a complex Gaussian, R-diagonal phases removed."""
    z = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    ph = np.diag(r) / np.abs(np.diag(r))
    return q * ph[None, :]


def tebd_inputs(nbonds: int = 256, seed: int = DEFAULT_SEED, chi_lo: int = 16, chi_hi: int = 512,
                d: int = 2):
    """Per bond: chi_i, A_i[chi,d,chi], B_i[chi,d,chi] (complex64), G_i[d,d,d,d] (complex64).

    G_i[s1, s2, t1, t2] is the 4x4 unitary U[(s1 s2), (t1 t2)].
    """
    rng = np.random.default_rng(seed)
    chis = rng.integers(chi_lo, chi_hi + 1, size=nbonds)
    A, B, G = [], [], []
    for c in chis:
        c = int(c)
        A.append((rng.standard_normal((c, d, c)) + 1j * rng.standard_normal((c, d, c))).astype(np.complex64))
        B.append((rng.standard_normal((c, d, c)) + 1j * rng.standard_normal((c, d, c))).astype(np.complex64))
        G.append(haar_unitary(d * d, rng).reshape(d, d, d, d).astype(np.complex64))
    return [int(c) for c in chis], A, B, G


def tfim_bond_hamiltonian(J: float = 1.0, g: float = 0.5) -> np.ndarray:
    """Two-site term h[(s1 s2), (t1 t2)] of the transverse-field Ising chain (the model of the
    paper's App. A): J on the diagonal for equal spins, -J for opposite ones, -g/2 between
    states that differ by one spin flip (so H = sum_bonds h = J sum ZZ - g sum X)."""
    h = np.diag([J, -J, -J, J]).astype(np.float64)
    for i, j in ((0, 1), (0, 2), (1, 0), (1, 3), (2, 0), (2, 3), (3, 1), (3, 2)):
        h[i, j] = -0.5 * g
    return h


def itebd_initial_state(chi: int, seed: int = DEFAULT_SEED, d: int = 2):
    """Random two-site unit cell as in App. A: Gamma_A, Gamma_B [chi, d, chi] and Lambda_A,
    Lambda_B [chi], entries uniform in [-1, 1) (numpy PCG64 from ``seed``)."""
    rng = np.random.default_rng(seed)
    gam = [rng.uniform(-1.0, 1.0, (chi, d, chi)) for _ in range(2)]
    lam = [rng.uniform(-1.0, 1.0, chi) for _ in range(2)]
    return gam, lam


def heavy_hex_graph(rows: int = 4, cols: int = 9):
    """A heavy-hex patch: a brick-wall lattice of rows x cols degree-<=3 vertices (horizontal bonds
    along each row, a vertical bond below (r, c) when r + c is even) with one extra degree-2 vertex
    inserted on every bond.  Returns (n_vertices, edges) with edges (u, v), u < v, in a fixed order."""
    def vid(r, c):
        return r * cols + c
    base = []
    for r in range(rows):
        for c in range(cols):
            if c + 1 < cols:
                base.append((vid(r, c), vid(r, c + 1)))
            if r + 1 < rows and (r + c) % 2 == 0:
                base.append((vid(r, c), vid(r + 1, c)))
    n = rows * cols
    edges = []
    for u, v in base:
        edges.append((u, n))
        edges.append((v, n))
        n += 1
    return n, sorted((min(a, b), max(a, b)) for a, b in edges)


def bp_tns_inputs(n: int, edges, chi: int, seed: int = DEFAULT_SEED, d: int = 2):
    """Random real TNS on a graph for belief propagation: site tensor V_i[s, b_1 .. b_k] with d
    physical states and one bond of dimension chi per neighbour (neighbours in ascending order),
    entries standard normal; messages M_{i->j} start as the identity / sqrt(chi) (unit Frobenius
    norm).  Messages are listed per edge e = (u, v): index 2e is u->v, 2e + 1 is v->u."""
    rng = np.random.default_rng(seed)
    deg = [0] * n
    for u, v in edges:
        deg[u] += 1
        deg[v] += 1
    V = [rng.standard_normal((d,) + (chi,) * deg[i]) for i in range(n)]
    M = [np.eye(chi) / np.sqrt(chi) for _ in range(2 * len(edges))]
    return V, M


def complex_heff_inputs(chi: int, seed: int = DEFAULT_SEED, chi_r: int | None = None, Dw: int = 3, d: int = 2):
    """Complex H_eff inputs: psi[chi,d,d,chi_r], L[chi,Dw,chi], R[chi_r,Dw,chi_r], W[Dw,Dw,d,d],
    complex128 with N(0,1) real and imaginary parts (numpy PCG64 from ``seed``)."""
    chi_r = chi if chi_r is None else chi_r
    rng = np.random.default_rng(seed)
    c = lambda *s: rng.standard_normal(s) + 1j * rng.standard_normal(s)
    return c(chi, d, d, chi_r), c(chi, Dw, chi), c(chi_r, Dw, chi_r), c(Dw, Dw, d, d)


def hermitian_heff_inputs(chi: int, seed: int = DEFAULT_SEED, chi_r: int | None = None):
    """Complex environments that make the Heisenberg H_eff Hermitian: L, R complex128 with
    L_w <- (L_w + conj(L_{sigma(w)})^T)/2 (the complex form of the channel-wise symmetrisation),
    W the real Heisenberg MPO as complex128, psi complex128; all parts N(0,1)."""
    chi_r = chi if chi_r is None else chi_r
    rng = np.random.default_rng(seed)
    c = lambda *s: rng.standard_normal(s) + 1j * rng.standard_normal(s)
    herm = lambda E: 0.5 * (E + np.conj(np.transpose(E, (2, 1, 0))[:, MPO_SIGMA, :]))
    psi, L, R = c(chi, 2, 2, chi_r), herm(c(chi, 5, chi)), herm(c(chi_r, 5, chi_r))
    return psi, L, R, heisenberg_mpo().astype(np.complex128)
