"""Plain PyTorch formulas of the objectives that gradients are taken of (reference for the
library's qlga_objective in the tests; autograd gives the reference cotangents).  State tensors
(5, ny, nx, 2, 2): level m = +2..-2, y, x, qubit (a, b), (re, im); psi = a + b."""
import math


def population(x, level):
    """sum |a_m|^2 + |b_m|^2 of level index `level`."""
    return (x[level] * x[level]).sum()


def _psi(x):
    return x[:, :, :, 0, 0] + x[:, :, :, 1, 0], x[:, :, :, 0, 1] + x[:, :, :, 1, 1]


def _theta(pr, pi):
    """psi^T J psi = 2 psi_2 psi_-2 - 2 psi_1 psi_-1 + psi_0^2 (re, im) per site."""
    def prod(i, j):
        return pr[i] * pr[j] - pi[i] * pi[j], pr[i] * pi[j] + pi[i] * pr[j]
    r20, i20 = prod(0, 4)
    r11, i11 = prod(1, 3)
    r00, i00 = prod(2, 2)
    return 2 * r20 - 2 * r11 + r00, 2 * i20 - 2 * i11 + i00


def singlet_fraction(x):
    pr, pi = _psi(x)
    rho = (pr * pr + pi * pi).sum(0)
    tr, ti = _theta(pr, pi)
    return (tr * tr + ti * ti).sum() / (rho * rho).sum()


def energy(x, g):
    """sum over sites of sum_axis sum_m |psi_m(j+1) - psi_m(j)|^2 (periodic forward differences)
    + g0/2 rho^2 + g1/2 |F|^2 + g2/10 |psi^T J psi|^2."""
    pr, pi = _psi(x)
    grad = 0.0
    for dim in (2, 1):
        if x.shape[dim] > 1:
            grad = grad + ((pr.roll(-1, dims=dim) - pr) ** 2 + (pi.roll(-1, dims=dim) - pi) ** 2).sum()
    n2 = pr * pr + pi * pi
    rho = n2.sum(0)
    Fz = 2 * (n2[0] - n2[4]) + (n2[1] - n2[3])
    r = math.sqrt(1.5)

    def cc(i, j):  # conj(psi_i) psi_j
        return pr[i] * pr[j] + pi[i] * pi[j], pr[i] * pi[j] - pi[i] * pr[j]
    terms = [cc(0, 1), cc(1, 2), cc(2, 3), cc(3, 4)]
    w = (1.0, r, r, 1.0)
    Fpr = 2 * sum(wk * t[0] for wk, t in zip(w, terms))
    Fpi = 2 * sum(wk * t[1] for wk, t in zip(w, terms))
    F2 = Fz * Fz + Fpr * Fpr + Fpi * Fpi
    tr, ti = _theta(pr, pi)
    g0, g1, g2 = g[0], g[1], g[2]
    return grad + (0.5 * g0 * rho * rho + 0.5 * g1 * F2 + 0.1 * g2 * (tr * tr + ti * ti)).sum()
