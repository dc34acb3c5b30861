"""Helpers shared by the GPU tests: numpy (4, rows, cols) arrays <-> device tensors."""
import numpy as np
import torch

from paper_2507_13731_gb300 import qlr

TORCH_DT = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}


def dev_rowmajor(a: np.ndarray, dt: str = "f32", pure: bool = False) -> torch.Tensor:
    t = torch.from_numpy(np.ascontiguousarray(a[1:] if pure else a)).to(TORCH_DT[dt])
    return t.cuda().contiguous()


def dev_thin(a: np.ndarray, dt: str = "f32") -> torch.Tensor:
    t = torch.from_numpy(np.ascontiguousarray(a)).to(TORCH_DT[dt]).cuda()
    return qlr.to_thin(t)


def host(t: torch.Tensor) -> np.ndarray:
    x = t.detach().float().cpu().double().numpy() if t.dtype == torch.bfloat16 else t.detach().cpu().double().numpy()
    if x.shape[0] == 3:
        x = np.concatenate([np.zeros((1,) + x.shape[1:]), x])
    return x


def small(l: int, k: int | None = None) -> torch.Tensor:
    """FP64 small-matrix buffer (4 planes, column-major l x k): shape (4, k, l) in memory."""
    return torch.zeros(4, k if k is not None else l, l, dtype=torch.float64, device="cuda")


def small_to_np(t: torch.Tensor) -> np.ndarray:
    """(4, cols, rows) storage -> (4, rows, cols) numpy."""
    return t.detach().cpu().numpy().transpose(0, 2, 1).copy()


def np_to_small(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a.transpose(0, 2, 1))).cuda()
