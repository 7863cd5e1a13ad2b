"""QUEEN's per-frame residual-training hot path (arXiv 2412.04469) on GB300:
the C-ABI library libqueen_gb300.so (include/queen.h), its ctypes binding
(binding.py), device buffers and the training iteration (pipeline.py), the
autograd Functions (autograd.py) and the streaming trainer with the learned
static skip (sequence.py)."""
