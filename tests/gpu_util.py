"""Helpers for the GPU tests: move column-major data and pack varlen batches."""
from __future__ import annotations

import numpy as np

from paper_2608_25469_gb300 import build as _build


def lib():
    _build.build()
    from paper_2608_25469_gb300 import hsma
    return hsma


def torch_dtype(np_dtype):
    import torch
    return {np.float64: torch.float64, np.complex128: torch.complex128, np.float32: torch.float32,
            np.complex64: torch.complex64}[np.dtype(np_dtype).type]


class Batch:
    """A varlen batch packed into two device buffers, plus device pointer/size arrays."""

    def __init__(self, As, Bs, device="cuda"):
        import torch
        self.batch = len(As)
        self.dtype = As[0].dtype if As else np.float64
        es = np.dtype(self.dtype).itemsize
        self.m = np.array([a.shape[1] for a in As], dtype=np.int32)
        self.n = np.array([b.shape[1] for b in Bs], dtype=np.int32)
        self.lda = np.array([max(1, a.shape[0]) for a in As], dtype=np.int32)
        self.ldb = np.array([max(1, b.shape[0]) for b in Bs], dtype=np.int32)
        sizeA = np.array([a.size for a in As], dtype=np.int64)
        sizeB = np.array([b.size for b in Bs], dtype=np.int64)
        self.offA = np.concatenate([[0], np.cumsum(sizeA)[:-1]]) if self.batch else np.zeros(0, np.int64)
        self.offB = np.concatenate([[0], np.cumsum(sizeB)[:-1]]) if self.batch else np.zeros(0, np.int64)
        hostA = np.concatenate([np.asarray(a, dtype=self.dtype).ravel(order="F") for a in As]) if self.batch else np.zeros(1, self.dtype)
        hostB = np.concatenate([np.asarray(b, dtype=self.dtype).ravel(order="F") for b in Bs]) if self.batch else np.zeros(1, self.dtype)
        self.dA = torch.from_numpy(hostA).to(device)
        self.dB = torch.from_numpy(hostB).to(device)
        baseA, baseB = self.dA.data_ptr(), self.dB.data_ptr()
        ptrA = (baseA + self.offA * es).astype(np.int64)
        ptrB = (baseB + self.offB * es).astype(np.int64)
        self.d_ptrA = torch.from_numpy(ptrA).to(device)
        self.d_ptrB = torch.from_numpy(ptrB).to(device)
        self.d_m = torch.from_numpy(self.m).to(device)
        self.d_n = torch.from_numpy(self.n).to(device)
        self.d_lda = torch.from_numpy(self.lda).to(device)
        self.d_ldb = torch.from_numpy(self.ldb).to(device)
        self.d_status = torch.zeros(1, dtype=torch.int32, device=device)
        self.shapesB = [b.shape for b in Bs]

    def args(self):
        return (self.d_m.data_ptr(), self.d_n.data_ptr(), self.d_ptrA.data_ptr(), self.d_lda.data_ptr(),
                self.d_ptrB.data_ptr(), self.d_ldb.data_ptr())

    def results(self):
        hostB = self.dB.cpu().numpy()
        out = []
        for b in range(self.batch):
            ld, cols = self.shapesB[b]
            out.append(hostB[self.offB[b]:self.offB[b] + ld * cols].reshape((ld, cols), order="F"))
        return out

    def status(self) -> int:
        return int(self.d_status.cpu().numpy()[0])
