"""PHSVDS hot path on GB300: C-ABI library binding (lazy) and input generators."""
