"""Seeded synthetic inputs: P1 FE eigenproblems and their AMG hierarchies."""
