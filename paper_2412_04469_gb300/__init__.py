"""QUEEN residual-training hot path on GB300 (placeholder, filled in below)."""
