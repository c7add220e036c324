"""Gauge-covariant convolutional network used as a learned smoother (oracle).

The paper does not have this part; the workload asks for a small
gauge-covariant convolutional network, trained on the solver's own residual /
error pairs, that stands in for the smoother.  The layer restated here:

  phi[o](x) = sum_c sum_h W[h][o][c] (T_h psi[c])(x),

with hops h = 0 (identity), 1 + 2 mu (T psi(x) = U_mu(x) psi(x + mu)) and
2 + 2 mu (T psi(x) = U_mu(x - mu)^H psi(x - mu)), the fermion time-boundary
sign on hops across t = Lt-1 -> 0, and W[h][o][c] a complex 4x4 matrix acting
on the spin index.  Colour is only touched by the parallel transport, so the
layer is gauge covariant: psi -> g psi, U_mu(x) -> g(x) U_mu(x) g(x+mu)^H
gives phi -> g phi.  The network is three such layers without bias or
nonlinearity, channels 1 -> C -> C -> 1, N(r) = L3 L2 L1 r.

Training loss for one residual r: L = ||r - D N(r)||^2 / ||r||^2.  With the
error e = D^{-1} r this is ||N(r) - e||^2 in the D^H D norm, so residual /
error pairs enter through r alone.  Gradients (Wirtinger, dL/dz*):
  G3 = dL/dN* = -D^H (r - D N(r)) / ||r||^2,
  dL/dpsi*   = L^H G  with L^H: hop h -> reversed hop, W -> W^H,
  dL/dW[h][o][c]* = sum_x sum_colour G[o](x) (T_h psi[c])(x)^H  (4x4 spin),
and for the real and imaginary parts A, B of W: dL/dA = 2 Re dL/dW*,
dL/dB = 2 Im dL/dW*.
"""
import numpy as np

from .dirac import _axis, _field, shift_backward, shift_forward

REVERSE = [0, 2, 1, 4, 3, 6, 5, 8, 7]  # hop h <-> its reverse


def transport(psi, U, dims, h):
    """T_h psi for one spinor field psi (V*12,) -> (V*12,)."""
    if h == 0:
        return np.array(psi, dtype=np.complex128)
    mu = (h - 1) // 2
    f = _field(psi, dims, (4, 3))
    Uf = _field(U, dims, (4, 3, 3))[..., mu, :, :]
    if h % 2 == 1:  # forward
        out = np.einsum('...ab,...sb->...sa', Uf, shift_forward(f, mu))
    else:
        Ub = np.roll(Uf, 1, axis=_axis(mu))
        out = np.einsum('...ba,...sb->...sa', Ub.conj(), shift_backward(f, mu))
    return out.reshape(-1)


def spin_mix(Wm, psi):
    """(Wm psi)_{s,a} = sum_s' Wm[s,s'] psi_{s',a} at every site."""
    f = np.asarray(psi).reshape(-1, 4, 3)
    return np.einsum('st,vta->vsa', Wm, f).reshape(-1)


def layer_forward(W, psi, U, dims):
    """W: (9, Cout, Cin, 4, 4); psi: (Cin, V*12) -> (Cout, V*12)."""
    _, Cout, Cin = W.shape[:3]
    out = np.zeros((Cout, psi.shape[1]), dtype=np.complex128)
    for c in range(Cin):
        for h in range(9):
            t = transport(psi[c], U, dims, h)
            for o in range(Cout):
                out[o] += spin_mix(W[h, o, c], t)
    return out


def layer_adjoint(W, g, U, dims):
    """L^H g: g (Cout, V*12) -> (Cin, V*12)."""
    _, Cout, Cin = W.shape[:3]
    out = np.zeros((Cin, g.shape[1]), dtype=np.complex128)
    for o in range(Cout):
        for h in range(9):
            t = transport(g[o], U, dims, REVERSE[h])
            for c in range(Cin):
                out[c] += spin_mix(W[h, o, c].conj().T, t)
    return out


def layer_weight_grad(g, psi, U, dims, Cout, Cin):
    """dL/dW* for the layer with input psi and output gradient g."""
    gW = np.zeros((9, Cout, Cin, 4, 4), dtype=np.complex128)
    for c in range(Cin):
        for h in range(9):
            t = transport(psi[c], U, dims, h).reshape(-1, 4, 3)
            for o in range(Cout):
                gW[h, o, c] = np.einsum('vsa,vta->st', g[o].reshape(-1, 4, 3), t.conj())
    return gW


def network_forward(Ws, r, U, dims):
    """activations [r, a1, a2, N(r)] for one residual r (V*12,)."""
    acts = [np.asarray(r, dtype=np.complex128)[None, :]]
    for W in Ws:
        acts.append(layer_forward(W, acts[-1], U, dims))
    return acts


def loss_and_grads(Ws, r, U, dims, apply_D, apply_DH):
    """L and dL/dW* of every layer for one residual."""
    acts = network_forward(Ws, r, U, dims)
    out = acts[-1][0]
    rn2 = np.vdot(r, r).real
    v = r - apply_D(out)
    L = np.vdot(v, v).real / rn2
    g = (-apply_DH(v) / rn2)[None, :]
    grads = [None] * len(Ws)
    for i in range(len(Ws) - 1, -1, -1):
        W = Ws[i]
        grads[i] = layer_weight_grad(g, acts[i], U, dims, W.shape[1], W.shape[2])
        g = layer_adjoint(W, g, U, dims)
    return L, grads


def init_weights(C, diag_scale, seed, noise=0.01):
    """Start close to a Jacobi step: channel 0 carries r through the network
    and is scaled by diag_scale; all other weights small random."""
    rng = np.random.default_rng(seed)
    shapes = [(9, C, 1, 4, 4), (9, C, C, 4, 4), (9, 1, C, 4, 4)]
    Ws = []
    for shp in shapes:
        W = noise * (rng.standard_normal(shp) + 1j * rng.standard_normal(shp)) / np.sqrt(2.0)
        W[0, 0, 0] += np.eye(4)
        Ws.append(W)
    Ws[2][0, 0, 0] *= diag_scale
    return Ws
