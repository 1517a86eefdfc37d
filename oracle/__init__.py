"""CPU oracle of the screened-WKB method (test infrastructure only)."""
