"""One-vs-one multiclass SVC on a precomputed quantum kernel (host orchestration).

The paper trains a support vector classifier on the simulated kernel matrix
(Sec. 3.2, Sec. 4.2 with 10-class MNIST / Fashion-MNIST).  Every class pair
(a, b) becomes a binary problem on the training points of a and b (labels +1 for
a, -1 for b); qsvm_svc_fit solves all pairs in one launch (one CTA per pair) and
qsvm_svc_decision evaluates all pairs' decision functions on a test x train
kernel; a test point gets one vote per pair and the class with most votes wins
(ties to the lower class).  This module only builds index lists and counts votes.
"""
from __future__ import annotations

from . import qsvm


class OneVsOneSVC:
    def __init__(self, C: float = 1.0, tol: float = 1e-8, max_iter: int = 10_000_000):
        self.C, self.tol, self.max_iter = C, tol, max_iter

    def fit(self, K, labels):
        """K: CUDA float64 (N, N) symmetric kernel; labels: CUDA int64 (N,)."""
        import torch
        self.classes = torch.unique(labels).tolist()
        self.pairs, self.problems = [], []
        for ia, a in enumerate(self.classes):
            for b in self.classes[ia + 1:]:
                idx = torch.nonzero((labels == a) | (labels == b)).flatten().to(torch.int64).contiguous()
                y = torch.where(labels[idx] == a, 1, -1).to(torch.int8).contiguous()
                alpha = torch.empty(idx.numel(), dtype=torch.float64, device=K.device)
                self.pairs.append((a, b))
                self.problems.append({"idx": idx, "y": y, "alpha": alpha})
        self.b, self.iters = qsvm.qsvm_svc_fit(K, self.problems, self.C, self.tol, self.max_iter)
        return self

    def decision(self, Kx):
        """Kx: CUDA float64 (M, N) test x train kernel -> (M, n_pairs) decision values."""
        return qsvm.qsvm_svc_decision(Kx, self.problems, self.b)

    def predict(self, Kx):
        import torch
        F = self.decision(Kx)
        votes = torch.zeros((Kx.shape[0], len(self.classes)), dtype=torch.int64, device=Kx.device)
        cls = {c: k for k, c in enumerate(self.classes)}
        for p, (a, b) in enumerate(self.pairs):
            win_a = F[:, p] > 0
            votes[:, cls[a]] += win_a.to(torch.int64)
            votes[:, cls[b]] += (~win_a).to(torch.int64)
        best = torch.argmax(votes, dim=1)  # first maximum: ties go to the lower class
        return torch.tensor(self.classes, device=Kx.device)[best]
