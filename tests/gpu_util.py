"""Helpers for the GPU tests: numpy <-> torch device buffers with exact bit patterns."""
import numpy as np

_TORCH_OF = {
    np.uint8: "uint8", np.int8: "int8", np.int16: "int16", np.uint16: "int16",
    np.int32: "int32", np.uint32: "int32", np.int64: "int64", np.uint64: "int64",
    np.float32: "float32",
}


def dev(a: np.ndarray):
    import torch
    a = np.ascontiguousarray(a)
    t = getattr(torch, _TORCH_OF[a.dtype.type])
    view = a.view(np.dtype(str(t).replace("torch.", "")))
    return torch.from_numpy(view.copy()).cuda()


def empty(shape, dtype):
    import torch
    t = getattr(torch, _TORCH_OF[np.dtype(dtype).type])
    return torch.empty(shape, dtype=t, device="cuda")


def host(t, dtype):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy().view(dtype)


def f32(x):
    return np.float32(x)


def compact(buf: np.ndarray, off: np.ndarray, lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    """Cells of a ragged buffer laid out with per-pixel block starts `off` (the GPU layout, blocks
    rounded up to a multiple of 4 cells) gathered into the compact order (no gaps)."""
    w = (hi.astype(np.int64) - lo.astype(np.int64) + 1).reshape(-1)
    start = np.repeat(off[:-1].astype(np.int64), w)
    pos = np.arange(int(w.sum()), dtype=np.int64) - np.repeat(np.concatenate([[0], np.cumsum(w)[:-1]]), w)
    return buf[start + pos]


def padded_offsets(lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    """Block starts of the GPU layout: exclusive scan of the window lengths rounded up to 4."""
    w = (hi.astype(np.int64) - lo.astype(np.int64) + 1).reshape(-1)
    return np.concatenate([[0], np.cumsum((w + 3) & ~3)]).astype(np.uint32)
