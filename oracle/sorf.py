"""Random-feature maps, plain FP64 definition (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

RFF section: z(x) = sqrt(2/N_F) [cos(w_1^T x + b_1), ..., cos(w_NF^T x + b_NF)],
W_RFF = G / sigma with G standard normal and b ~ U[0, 2 pi].

SORF section: W_SORF = (sqrt(d)/sigma) [H D_i]_{N_transform}, with D_i
Rademacher diagonals and H the Walsh-Hadamard matrix of the Sylvester
recursion H_{2^n} = [[H_{2^{n-1}}, H_{2^{n-1}}], [H_{2^{n-1}}, -H_{2^{n-1}}]],
H_1 = 1. For N_F > d the transform is repeated N_F/d times with independent
diagonals and the outputs concatenated.

Reading of the normalisation: each factor is the
orthogonal matrix H/sqrt(d) times D, so the product Q is orthogonal and the
rows of one stack of W have norm sqrt(d)/sigma, which is the scalar that the
SORF section substitutes for the chi-distributed S. Factor t uses D_{s,t}
and the sign flip is applied before H. The matrices are built densely here;
the fast transform is the CUDA side's business.
"""
from __future__ import annotations

import math

import numpy as np
import torch


def hadamard(d: int) -> np.ndarray:
    """Walsh-Hadamard matrix of order d = 2^n by the Sylvester recursion."""
    if d < 1 or d & (d - 1):
        raise ValueError("d must be a power of two")
    H = np.ones((1, 1))
    while H.shape[0] < d:
        H = np.block([[H, H], [H, -H]])
    return H


def sorf_matrix(signs: np.ndarray, sigma: float) -> np.ndarray:
    """Dense W [n_stack * d, d] from Rademacher signs [n_stack, T, d]."""
    n_stack, T, d = signs.shape
    Hn = hadamard(d) / math.sqrt(d)
    blocks = []
    for s in range(n_stack):
        Q = np.eye(d)
        for t in range(T):
            Q = Hn @ np.diag(signs[s, t].astype(np.float64)) @ Q
        blocks.append(math.sqrt(d) / sigma * Q)
    return np.concatenate(blocks, axis=0)


def rff_matrix(G: np.ndarray, sigma: float) -> np.ndarray:
    """W_RFF = G / sigma."""
    return np.asarray(G, dtype=np.float64) / sigma


def features(x, W, b):
    """z = sqrt(2/N_F) cos(x W^T + b) for rows x [N, d]; works on numpy or torch."""
    n_f = W.shape[0]
    if isinstance(x, torch.Tensor):
        Wt = torch.as_tensor(W, dtype=x.dtype)
        bt = torch.as_tensor(b, dtype=x.dtype)
        return math.sqrt(2.0 / n_f) * torch.cos(x @ Wt.T + bt)
    return math.sqrt(2.0 / n_f) * np.cos(np.asarray(x) @ np.asarray(W).T + np.asarray(b))


def gaussian_kernel(x: np.ndarray, y: np.ndarray, sigma: float) -> float:
    """The kernel the feature maps approximate: exp(-|x - y|^2 / (2 sigma^2))."""
    return float(np.exp(-np.sum((x - y) ** 2) / (2.0 * sigma * sigma)))
