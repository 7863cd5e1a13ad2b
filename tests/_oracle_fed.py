"""The oracle's compositing fed the GPU's own FP32 projection.

The FP64 oracle can project a scene itself, but then every projection
decision that FP32 could flip (a rect edge, a radius, the near plane) has to
be excluded from the comparison.  Fed the GPU's FP32 records and rects,
converted to double, the oracle composites exactly the tile lists the GPU
composites: its depth order is the GPU's stable (depth bits, index) order,
so the only decisions left to FP32 are the alpha threshold and cap and the
termination product, which the oracle flags per pixel.
"""
import numpy as np


def proj_from_gpu(splats, rects, n, width, height):
    """Oracle projection dict from the GPU's [n][12] splat records and
    [n][4] rects (x0, y0, x1, y1), as numpy arrays."""
    sp = np.asarray(splats, np.float32)[:n].astype(np.float64)
    rc = np.asarray(rects, np.int32)[:n]
    nonempty = (rc[:, 2] > rc[:, 0]) & (rc[:, 3] > rc[:, 1])
    return dict(mean2d=np.ascontiguousarray(sp[:, 0:2].T), opac=np.ascontiguousarray(sp[:, 2]),
                depth=np.ascontiguousarray(sp[:, 3]), conic=np.ascontiguousarray(sp[:, 4:7].T),
                rgb=np.ascontiguousarray(sp[:, 8:11].T), rect=np.ascontiguousarray(rc.T),
                radius=nonempty.astype(np.int32), fragile=np.zeros(n, np.int32),
                frag_rect=np.zeros((4, n), np.int32), width=int(width), height=int(height))
