"""Seeded synthetic inputs: detector geometry, pixel events and cut tables.

This package is the only code shared by the oracle side and the CUDA side; it
produces inputs and configuration constants and contains none of the seeding or
fitting arithmetic."""
