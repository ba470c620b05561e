"""Exact CPU oracle for Radic's determinant (test infrastructure only; see radic_oracle)."""
from .radic_oracle import *  # noqa: F401,F403
